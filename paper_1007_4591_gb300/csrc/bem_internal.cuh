// Internal declarations of libbem (not part of the public C ABI).
//
// Data layout in HBM (all arrays device-resident, owned by the mesh):
//   * panels, quadrature points and charges are each sorted by their own
//     63-bit Morton key (21 bits per axis, root cube shared by all sets);
//   * every point record stores its coordinates relative to the centre of
//     the leaf cell that contains it (FP32 float4 or FP64 double4, .w holds
//     the weight A_j w_q or the charge), so near-field differences never see
//     the absolute coordinate magnitude;
//   * multipole / local expansions are (p+1)^2 reals per cell in the compact
//     real layout  [n^2] = Re X_n^0,  [n^2 + 2m - 1] = Re X_n^m,
//     [n^2 + 2m] = Im X_n^m  (m = 1..n), scaled by the cell size so that every
//     translation operator is level independent.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <stdint.h>
#include <stdexcept>
#include <string>
#include <memory>
#include <vector>

#include "../../include/bem.h"

namespace bem {

constexpr int MAXP = 16;           // largest expansion order built
constexpr int MORTON_BITS = 21;    // bits per axis in a key
// M2L offset classes of a tree whose cells interact once separated by `ws`
// cells (ws = 1: children of the parent's neighbours not adjacent, offsets
// in [-3,3]^3 -> 343 classes; ws = 2: offsets in [-5,5]^3 -> 1331 classes)
inline int m2l_radius(int ws) { return 2 * ws + 1; }
inline int m2l_classes(int ws) { const int w = 2 * m2l_radius(ws) + 1; return w * w * w; }
constexpr double PI = 3.14159265358979323846;
constexpr double FOUR_PI = 12.566370614359172953850573533118;
constexpr double KCAL = 332.0637;  // e^2/(4 pi eps0 A) in kcal/mol

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string &msg);

#define BEM_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            throw ::bem::Error(e_ == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA,  \
                               std::string(#call) + ": " + cudaGetErrorString(e_) + " (" + \
                                   __FILE__ + ":" + std::to_string(__LINE__) + ")");      \
    } while (0)

#define BEM_CHECK_LAUNCH() BEM_CUDA(cudaGetLastError())

// Wall time of each build step (the stream synchronised at each mark),
// printed to stderr when the environment sets BEM_TIMING=1.
struct StepTimer {
    cudaStream_t s;
    bool on;
    std::chrono::steady_clock::time_point t;
    explicit StepTimer(cudaStream_t st) : s(st), on(false) {
        const char *e = std::getenv("BEM_TIMING");
        on = e && e[0] == '1';
        t = std::chrono::steady_clock::now();
    }
    void mark(const char *what) {
        if (!on) return;
        cudaStreamSynchronize(s);
        const auto n = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[bem] %-52s %9.1f ms\n", what, std::chrono::duration<double, std::milli>(n - t).count());
        t = n;
    }
};

// Raise a kernel's dynamic shared-memory limit once per (kernel, device);
// repeated requests are free (no runtime call), which keeps graph capture clean.
void ensure_smem_attr(const void *func, size_t bytes);

// ------------------------------------------------------- device array (RAII)
// Device memory held by the library's arrays, process-wide.  With a cap set
// (bem_set_device_memory_cap) an allocation beyond it fails with BEM_ENOMEM
// before reaching the allocator.
void dev_mem_reserve(size_t bytes);
void dev_mem_unreserve(size_t bytes);

template <class T>
struct DArray {
    T *p = nullptr;
    size_t n = 0;
    DArray() = default;
    DArray(const DArray &) = delete;
    DArray &operator=(const DArray &) = delete;
    DArray(DArray &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DArray &operator=(DArray &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DArray() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        dev_mem_reserve(count * sizeof(T));
        const cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            dev_mem_unreserve(count * sizeof(T));
            cudaGetLastError();
            throw ::bem::Error(e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA,
                               std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        n = count;
    }
    void release() {
        if (p) {
            cudaFree(p);
            dev_mem_unreserve(n * sizeof(T));
        }
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
    operator T *() const { return p; }
};

// ------------------------------------------------------------- structures
// Octree over one or more point sets sharing the root cube and leaf level.
struct Tree {
    int L = 0;                    // leaf level
    int ws = 1;                   // separation (in cells) of interacting cells: neighbours
                                  // are the leaves within ws cells, M2L partners lie farther
    std::vector<int> lvl_off;     // cells of level l: [lvl_off[l], lvl_off[l+1])
    int ncell = 0, nleaf = 0, leaf0 = 0;
    DArray<uint64_t> key;         // [ncell] Morton key at the cell's own level
    DArray<int4> ijk;             // [ncell] integer cell coordinates (x, y, z, level)
    DArray<int> parent;           // [ncell] (-1 at the root)
    DArray<int> child_beg;        // [ncell] first child (global index), -1 for leaves
    DArray<int> child_end;        // [ncell]
    DArray<int> cen_beg, qp_beg, chg_beg; // [nleaf+1] CSR of each sorted set over leaves
    bool has_cen = false, has_qp = false, has_chg = false;
    DArray<int> nbr_off, nbr;     // P2P: leaf -> adjacent leaves (incl. itself), CSR
    DArray<int> m2l_off, m2l_src, m2l_ofs; // per cell CSR: source cell, offset class
    int64_t nnbr = 0, nm2l = 0;
    int64_t p2p_pairs_cq = 0;     // (centroid target, quad source) pairs
    // translations grouped by operator for the batched dense form:
    // M2L pairs (out = target cell, in = source cell) sorted by offset class,
    // M2M pairs (out = parent, in = child) and L2L pairs (out = child,
    // in = parent) per child level, sorted by the child's octant.  A chunk is
    // (operator, first pair, pair count <= 64, 0).
    DArray<int> g_out, g_in;      // all grouped pairs: M2L, then M2M and L2L per level
    DArray<int4> g_chunk;
    DArray<int> p2p_order;        // leaves by decreasing near-field work (launch order)
    // near-field work lists in launch order, per source kind (quadrature
    // points, charges): two int4 of leaf data and nb records per CTA
    DArray<int4> p2p_hdr[2];
    DArray<int2> p2p_rec[2];
    int p2p_nb = 27;              // records per CTA (the most neighbour leaves)
    // P2M of the quadrature points as a product with fixed moments: the
    // points of each leaf grouped by panel into segments, and each segment's
    // multipole with unit density (its points' weights times their regular
    // solid harmonics) computed once; a product's P2M is then
    // M_leaf = sum over the leaf's segments of sigma(panel) x moment.
    DArray<int> p2m_seg_beg;      // [nleaf+1] the segments of each leaf (CSR)
    DArray<int> p2m_seg_panel;    // [nseg] panel of each segment
    DArray<float> p2m_seg_f;      // [nseg x cell stride] moments (mixed precision)
    DArray<double> p2m_seg_d;     // [nseg x cell stride] moments (FP64)
    int p2m_seg_p = -1;           // expansion order of the moments (-1: none built)
    DArray<int4> tc_super;        // tensor-core M2L work items (offset, first chunk, chunks)
    int tc_nsuper = 0;
    int m2l_chunk0 = 0, m2l_nchunk = 0;
    std::vector<int> m2m_chunk0, m2m_nchunk, l2l_chunk0, l2l_nchunk; // indexed by child level
    size_t bytes() const;
};

// Device-side view of a tree, passed to kernels by value.
struct TreeView {
    int L, ncell, nleaf, leaf0;
    const int4 *ijk;
    const int *parent, *child_beg, *child_end;
    const int *cen_beg, *qp_beg, *chg_beg;
    const int *nbr_off, *nbr;
    const int *m2l_off, *m2l_src, *m2l_ofs;
    const int *p2p_order;
    // per-panel P2M moments of the quadrature points (null: none)
    const int *seg_beg, *seg_panel;
    const float *seg_f;
    const double *seg_d;
    int seg_p;
};

TreeView view(const Tree &t);

// Source and target kinds of one fast multipole pass.
enum SrcKind { SRC_QUAD = 0, SRC_CHARGE = 1, SRC_DIPOLE = 2 };
// targets: normal field at the centroids (collocation), potential at the
// charges, potential at the quadrature points, normal field at the
// quadrature points with their panel's normal (Galerkin rows)
enum TgtKind { TGT_CEN_DN = 0, TGT_CHG_PHI = 1, TGT_QUAD_PHI = 2, TGT_QUAD_DN = 3 };

struct Mesh;

// Expansion/translation tables of one expansion order and precision, shared
// by every mesh of the device (built once per (device, p, precision)).
//   Rm2m: solid harmonics R_k^l of the 8 child offsets, full m range;
//   If:   irregular harmonics I_n^m (n <= 2p) of the 343 offset classes;
//   Om2l, Om2m, Ol2l: the translations as real (p+1)^2 x (p+1)^2 matrices
//         in the compact real layout, stored column-major ([in][out]) with
//         each [in] row padded with zeros to the cell stride.
struct Tables {
    int p = 0;
    int ws = 1;                   // the M2L operators cover the offset classes of this separation
    DArray<float> Rm2m_f, If_f, Om2l_f, Om2m_f, Ol2l_f;
    DArray<double> Rm2m_d, If_d, Om2l_d, Om2m_d, Ol2l_d;
    DArray<float> Tc_f;           // M2L operators in FP32, tensor-core tile order (the kernel
                                  // splits them into their TF32 hi / lo parts as it loads them)
    size_t bytes() const {
        return Tc_f.bytes() + Rm2m_f.bytes() + If_f.bytes() + Om2l_f.bytes() + Om2m_f.bytes() + Ol2l_f.bytes() +
               Rm2m_d.bytes() + If_d.bytes() + Om2l_d.bytes() + Om2m_d.bytes() + Ol2l_d.bytes();
    }
};

struct Timers {
    bool on = false;
    // the last timed product ran its near field before L2P (the epilogue
    // fused into L2P): events 4-5 bracket P2P and 5-6 L2P
    bool near_before_l2p = false;
    cudaEvent_t ev[8] = {};
    double ms[7] = {};
    cudaEvent_t kev[4] = {};  // inside the tensor-core M2L stage: split | kernel | (unused)
    cudaEvent_t nev[3] = {};  // inside the near-field phase: strength records | near-field kernel
};

struct Mesh {
    bem_options opt;
    cudaStream_t stream = nullptr;     // the mesh's own non-blocking work stream
    cudaStream_t user = nullptr;       // the caller's stream (ordering hand-off)
    cudaEvent_t ev_enter = nullptr;
    cudaStream_t stream2 = nullptr;    // second work stream: near field next to the far field
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    long long wait_budget = 2000000000ll; // clock cycles a device-side pipeline wait may take
    // captured K' product on fixed buffers gx -> gy
    cudaGraphExec_t g_mv = nullptr;
    DArray<double> gx, gy;
    bool capturing = false;
    int device = 0;
    int64_t np = 0, nc = 0, nq = 0, nqp = 0;
    double eps_in = 1, eps_out = 80, ehat = 0;
    double root_min[3] = {0, 0, 0};
    double side = 1;
    int L = 0;
    double ms_build = 0;

    // sorted panels (targets / unknowns)
    DArray<int> cen_perm;        // sorted -> original panel
    DArray<double> cen64;        // [np][3] absolute centroid
    DArray<double> nrm64;        // [np][3]
    DArray<double> area64;       // [np]
    DArray<float4> cen32, nrm32; // relative centroid / normal (mixed precision)
    DArray<double4> cen64r, nrm64r; // relative centroid / normal (fp64 mode)
    // Galerkin form: each quadrature point's panel normal, in the quadrature
    // points' order (records as nrm32 / nrm64r, and absolute f64 [nqp][3])
    DArray<float4> nrmq32;
    DArray<double4> nrmq64r;
    DArray<double> nrmq64;
    DArray<double> gq_tmp;             // [nqp] Galerkin scratch (direct sums at the quadrature points)
    DArray<double> lamq;               // [nqp] Galerkin dipole moments of the transposed product / B_G^T
    DArray<double> ctq;                // [np] C^T q (sorted panels), valid when ctq_ok
    bool ctq_ok = false;
    DArray<uint64_t> cen_key;
    // sorted quadrature points (sources)
    DArray<int> qp_panel;        // sorted quad point -> sorted panel
    DArray<double> qpg64;        // [nqp][3] absolute coordinates
    DArray<double> qw64;         // [nqp] A_j w_q
    DArray<float4> qp32;         // (y_rel, A_j w_q)
    DArray<double4> qp64r;
    DArray<uint64_t> qp_key;
    // sorted charges
    DArray<int> chg_perm;        // sorted -> original charge
    DArray<double> chgg64;       // [nc][3] absolute coordinates
    DArray<double> q64;          // [nc] charge values (sorted order)
    DArray<float4> chg32;        // (x_rel, q)
    DArray<double4> chg64r;
    DArray<uint64_t> chg_key;

    Tree tp;   // panels (centroids + quadrature points): K' and K'^T
    Tree tc;   // panels + charges: B, C and the adjoint charge terms

    // near-singular FP64 table (CSR over sorted targets) and its transpose
    DArray<int> nt_off, nt_col, ntT_off, ntT_col;
    DArray<double> nt_val, ntT_val;
    bool ntT_ok = false;               // the transpose is built (on first use by K'^T)
    int64_t nt_nnz = 0;
    DArray<int> qp_of_panel;           // [np][nq] sorted quadrature points of each sorted panel

    std::shared_ptr<Tables> tab;       // translations of the panel tree (ws = 1)
    std::shared_ptr<Tables> tab2;      // of a charge tree separated by two cells (ws = 2)

    // expansion buffers (sized for the larger tree)
    DArray<float> Mf, Lf;
    DArray<double> Md, Ld;

    // work vectors
    DArray<double> xs, ys, zs;         // sorted-order f64 vectors
    DArray<double> near64;             // near field + 4 pi x near-singular table x (collocation product)
    // charge-panel pairs integrated exactly (BEM_FLAG_CHARGE_NEAR_EXACT):
    // panel vertices in sorted order, the (exact - rule) / (4 pi) of each pair's
    // potential and gradient by charge (CSR), and the potential part by panel
    DArray<double> pan64;              // [np][9]
    DArray<int> cn_off, cn_col, cnT_off, cnT_row;
    DArray<double> cn_val, cnT_val;    // [nnz][4], [nnz]
    int cn_nnz = 0;
    DArray<float4> str32;              // per-pass near-field source strength records (mixed)
    DArray<double4> str64;             // (fp64 mode)
    DArray<float> far_f, near_f;       // per-target partial results (mixed)
    DArray<double> far_d, near_d;      // (fp64 mode)
    DArray<double> io_a, io_b;         // staging for host or unsorted arguments
    DArray<double> red;                // reduction scratch
    DArray<float> Mtc;                 // multipoles split hi|lo for the tensor-core M2L
    DArray<float> dpart_f;             // direct-sum partials (mixed)
    DArray<double> dpart_d;            // direct-sum partials (fp64)
    double *h_pinned = nullptr;        // small pinned host buffer

    // GMRES workspace
    DArray<double> V, H, gv, cs, sn, yv, hv, part;
    // last solve (for the adjoint)
    DArray<double> sigma_s;
    bool have_sigma = false;

    DArray<int> dev_err;               // device error word (bounded waits that ran out)
    Timers tm;
    size_t bytes() const;
};

// --------------------------------------------------------------- helpers
inline int ncoef(int p) { return (p + 1) * (p + 1); }
// per-cell stride of the expansion arrays: (p+1)^2 rounded up to 4 values
inline int cell_stride(int p) { return ((p + 1) * (p + 1) + 3) & ~3; }
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// geometry + trees (bem_tree.cu)
void build_geometry_and_trees(Mesh &m, const double *d_panels, const double *d_charges);
void rebuild_charge_tree(Mesh &m, const double *d_charges);
// panels: [np][3][3] f64 device array in the caller's order (read when
// opt.near_table == BEM_NEAR_EXACT)
void build_near_table(Mesh &m, const double *panels);
// exact charge-panel pairs (bem_charge_near.cu): the panel vertices kept at
// creation, the table built per charge set, and its application to the
// potential (and gradient) at the charges (C s; stride / ncomp 1 / 1 or 4 / 4
// for (phi, grad)) and to C^T u (per panel); no-ops unless the flag is set
// Galerkin dipole moments lam_j w_q at every quadrature point (into m.lamq)
void galerkin_moments(Mesh &m, const double *lam);
bool charge_near_on(const Mesh &m);
void keep_panel_vertices(Mesh &m, const double *d_panels);
void build_charge_near(Mesh &m);
void charge_near_phi(Mesh &m, const double *s_sorted, double *out, int stride, int ncomp);
void charge_near_ct(Mesh &m, const double *u_sorted, double *v);
// per panel, its quadrature points' positions in the sorted quadrature order
void build_qp_of_panel(Mesh &m);
// the near-singular table's transpose (for K'^T), built on first use
void transpose_near_table(Mesh &m);
// Galerkin form: per-quadrature-point normal records and the scratch it needs
void build_galerkin_geometry(Mesh &m);
void build_tables(Mesh &m);
const Tables &tables_for(const Mesh &m, const Tree &t);
// stable sort of int keys in [0, 2^bits) with int values, on the device
void sort_pairs_int(const int *k_in, const int *v_in, int *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s);
// hand-written sorting and scans (bem_sort.cu): stable LSD radix sorts of
// the low `bits` bits of the keys (v_in / v_out may be null: keys only),
// exclusive / inclusive int scans, and the unique values of a sorted array
// (returns their count)
void radix_sort_u64(const uint64_t *k_in, const int *v_in, uint64_t *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s);
void radix_sort_u32(const uint32_t *k_in, const int *v_in, uint32_t *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s);
void scan_exclusive_i32(const int *in, int *out, int64_t n, cudaStream_t s);
void scan_inclusive_i32(const int *in, int *out, int64_t n, cudaStream_t s);
int64_t unique_sorted_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s);
// the per-panel P2M moments of a tree's quadrature points (bem_leaf.cu);
// nothing is built when BEM_FLAG_P2M_FROM_POINTS is set, when the tree has no
// far field or no quadrature points, or when the moments would take more than
// half of the free device memory (P2M then works from the points)
void build_p2m_moments(Mesh &m, Tree &t);
void build_translation_groups(Mesh &m, Tree &t);
// tensor-core M2L (bem_tc.cu)
bool tc_m2l_available(const Mesh &m);
void build_tc_tables(int p, const std::vector<double> &om2l, int nops, std::vector<float> &op);
void build_tc_super(Tree &t, const std::vector<int4> &chunks_m2l, cudaStream_t s);
void m2l_tc(Mesh &m, const Tree &t, const float *M, float *L, bool timed = false);
bool use_tc_m2l(const Mesh &m);
size_t tc_staging_floats(const Mesh &m);
void compute_bbox(const double *d, int64_t n, int stride, double *lo, double *hi, cudaStream_t s);

// fast multipole passes (bem_fmm.cu).  `dens` is indexed in sorted panel
// order for SRC_QUAD (strength A_j w_q dens[panel]) and sorted charge order for
// SRC_CHARGE (strength dens[k], or the stored q when dens is null).  The output
// `out` (sorted target order, f64) receives sum over sources of
//   TGT_CEN_DN : n_i . grad_{c_i} (s / (4 pi |c_i - y|))
//   TGT_CHG_PHI: s / (4 pi |x_k - y|)
void fmm_pass(Mesh &m, const Tree &t, SrcKind sk, TgtKind tk, const double *dens, double *out,
              bool timed);
// The collocation operator product y = x + Ehat (K' x + table x) (sorted
// order): the K' pass with its epilogue fused into the last kernel.
void kprime_apply(Mesh &m, const double *xs, double *ys);
// Transposed K' pass: out[j] = (K'^T lam)_j without the near-singular table
// (dipoles lam_i n_i at the collocation points, potential at the quadrature
// points, weighted sum over each panel's points).
void fmm_pass_t(Mesh &m, const double *lam, double *out);
bool is_near_field_kernel(const void *func);

// Products between the charges and the surface (B q, C sigma): the fast
// multipole pass on the charge tree, or the direct sum over all pairs,
// following opt.charge_mode.
void charge_pass(Mesh &m, SrcKind sk, TgtKind tk, const double *dens, double *out);
bool charge_direct(const Mesh &m);
void direct_pass(Mesh &m, SrcKind sk, TgtKind tk, const double *dens, double *out);
void build_ctq(Mesh &m);
double energy_from_ctq(Mesh &m, const double *sig_s);

// solver pieces (bem_solver.cu)
void matvec_sorted(Mesh &m, const double *xs, double *ys);
void matvec_t_sorted(Mesh &m, const double *xs, double *ys);
void exclusive_scan_int(const int *in, int *out, int n, cudaStream_t s);
void gather_f64(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s);
void scatter_f64(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s);
void scatter_rows3(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s);

}  // namespace bem
