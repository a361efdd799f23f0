// P2M (sources -> multipole of their leaf) and L2P (local expansion of a
// leaf -> its targets), Sec. 2.3, with the expansion order as a template
// parameter: fixing p at compile time turns the solid harmonic recurrence
// into straight-line code with folded constants.  P2M instantiates every
// order 1..MAXP, L2P the orders 6, 8, 10, 12 (other orders take the generic
// kernel).
#include <algorithm>

#include "bem_device.cuh"

namespace bem {

template <class KernelT>
static void leaf_smem(KernelT kern, size_t bytes) {
    if (bytes > 48 * 1024) ensure_smem_attr(reinterpret_cast<const void *>(kern), bytes);
}

// ------------------------------------------------------------------- P2M
// A CTA of 4 warps owns one leaf; each warp takes 32 points at a time.  The
// recurrence emits a point's (p+1)^2 real values in a fixed order (slot k:
// m = 0 values first, then the re / -im pairs column by column); every 32
// slots a warp's lanes have written one 32 x 32 block of its row buffer
// (stride 33: conflict-free both ways), and each lane adds up its column of
// the block over the 32 points in registers.  The warps' column sums are
// added in a fixed order at the end.  Lanes without a point write zeros.
constexpr int P2M_WARPS = 4;
constexpr int P2M_RS = 33;

// slot of R_n^m (re; im at +1) in the emission order, and its compact index
template <int P>
__host__ __device__ constexpr int p2m_slot(int n, int m) {
    return m == 0 ? n : (P + 1) + (m - 1) * (2 * P + 2 - m) + 2 * (n - m);
}
template <int P>
__device__ constexpr int p2m_compact(int k) {
    // inverse of p2m_slot, then the compact real layout (n^2, n^2 + 2m - 1 | n^2 + 2m)
    if (k <= P) return k * k;
    int m = 1;
    while (p2m_slot<P>(P, m) + 1 < k) ++m;
    const int off = k - p2m_slot<P>(m, m);
    const int n = m + off / 2;
    return n * n + 2 * m - 1 + (off & 1);
}

template <class T, int SRC, int P>
__global__ void __launch_bounds__(P2M_WARPS * 32)
k_p2m_c(TreeView tv, const typename V4T<T>::t *rec, const int *qpanel, const double *dens, int cs, T inv_h, T *M) {
    constexpr int NC = (P + 1) * (P + 1);
    constexpr int KC = (NC + 31) / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    // the first upward translation may start now (it waits for this grid's
    // results before it reads them)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T *buf = sm + (size_t)w * 32 * P2M_RS;
    T *row = buf + lane * P2M_RS;
    const int leaf = blockIdx.x;
    const int *beg = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int b = beg[leaf], e = beg[leaf + 1];
    T acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = 0;
    auto flush = [&](int chunk) {  // column `lane` of block `chunk`, summed over the 32 rows
        __syncwarp();
        if (32 * chunk + lane < NC) {
            T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                s0 += buf[j * P2M_RS + lane];
                s1 += buf[(j + 1) * P2M_RS + lane];
                s2 += buf[(j + 2) * P2M_RS + lane];
                s3 += buf[(j + 3) * P2M_RS + lane];
            }
#pragma unroll
            for (int k = 0; k < KC; ++k)
                if (k == chunk) acc[k] += (s0 + s1) + (s2 + s3);
        }
        __syncwarp();
    };
    auto put = [&](int k, T v) {
        row[k & 31] = v;
        if ((k & 31) == 31 || k == NC - 1) flush(k >> 5);
    };
    for (int base = b + w * 32; base < e; base += P2M_WARPS * 32) {
        const int i = base + lane;
        T x = 0, y = 0, z = 0, s = 0;
        if (i < e) {
            const typename V4T<T>::t r = rec[i];
            x = r.x * inv_h;
            y = r.y * inv_h;
            z = r.z * inv_h;
            s = src_strength<T, SRC>(r.w, i, qpanel, dens);
        }
        regular_solid_c<T, P>(x, y, z, [&](int n, int m, T re, T im) {
            const int k = p2m_slot<P>(n, m);
            put(k, s * re);
            if (m > 0) put(k + 1, -s * im);
        });
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        if (c < NC) sm[w * NC + c] = acc[k];
    }
    __syncthreads();
    T *out = M + (size_t)(tv.leaf0 + leaf) * cs;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = threadIdx.x + P2M_WARPS * 32 * k;
        if (c < NC) {
            T a = 0;
#pragma unroll
            for (int v = 0; v < P2M_WARPS; ++v) a += sm[v * NC + c];
            out[p2m_compact<P>(c)] = a;
        }
    }
}


// ------------------------------------------------------------------ launch
template <class T, int SRC, int P>
static void p2m_launch_c(const TreeView &tv, int nleaf, const typename V4T<T>::t *src, const int *qpanel,
                         const double *dens, int cs, T inv_h, T *M, cudaStream_t s) {
    constexpr int NC = (P + 1) * (P + 1);
    const size_t sm = std::max<size_t>((size_t)P2M_WARPS * 32 * P2M_RS, (size_t)P2M_WARPS * NC) * sizeof(T);
    auto kern = k_p2m_c<T, SRC, P>;
    leaf_smem(kern, sm);
    kern<<<nleaf, P2M_WARPS * 32, sm, s>>>(tv, src, qpanel, dens, cs, inv_h, M);
    BEM_CHECK_LAUNCH();
}

template <class T, int P = 1>
static void p2m_dispatch(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src,
                         const int *qpanel, const double *dens, int p, int cs, T inv_h, T *M, cudaStream_t s) {
    if constexpr (P <= MAXP) {
        if (p != P) return p2m_dispatch<T, P + 1>(tv, nleaf, sk, src, qpanel, dens, p, cs, inv_h, M, s);
        if (sk == SRC_QUAD) p2m_launch_c<T, SRC_QUAD, P>(tv, nleaf, src, qpanel, dens, cs, inv_h, M, s);
        else if (sk == SRC_CHARGE) p2m_launch_c<T, SRC_CHARGE, P>(tv, nleaf, src, qpanel, dens, cs, inv_h, M, s);
        else throw Error(BEM_EUNSUPPORTED, "P2M source kind not built");
    } else {
        throw Error(BEM_EINVAL, "expansion order out of range");
    }
}

// ------------------------------------------------- P2M from panel moments
// The quadrature points' strengths are s_i = w_i sigma(panel_i), so a leaf's
// multipole is sum over the panels j with points in the leaf of
// sigma_j (sum over those points of w_i conj R(y_i - z) / h^n): the inner sum
// (the segment's moment) depends on the geometry only.  The moments are
// built once per mesh with the point P2M above (every segment a CTA, unit
// density); a product's P2M then reads them (HBM bound) instead of running
// the recurrence for every point.

constexpr int P2M_SEG_MAXNC = 384;  // (p+1)^2 for p <= 18: three coefficients per thread

// one CTA per leaf: coefficient k of the leaf's multipole is the sum over its
// segments, in segment order, of sigma(panel) x moment_k.  A thread keeps
// P2M_SEG_BATCH moment loads in flight (a leaf has ~26 segments: about two
// batches), and the first batch is issued before the densities are gathered
// (two dependent loads), so the latencies overlap.
constexpr int P2M_SEG_BATCH = 16;

template <class T>
__global__ void __launch_bounds__(128)
k_p2m_seg(TreeView tv, const T *__restrict__ mom, const double *__restrict__ dens, int nc, int cs, T *M) {
    // the first upward translation may start now (it waits for this grid's
    // results before it reads them)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int NJ = P2M_SEG_MAXNC / 128, B = P2M_SEG_BATCH;
    __shared__ T s_sig[128];
    const int leaf = blockIdx.x;
    const int b = tv.seg_beg[leaf], e = tv.seg_beg[leaf + 1];
    T acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = 0;
    for (int s0 = b; s0 < e; s0 += 128) {
        const int ns = min(128, e - s0);
        const T *base = mom + (size_t)s0 * cs + threadIdx.x;
        T v[B];
        auto load = [&](int j, int q0) {
            const bool ok = (int)threadIdx.x + 128 * j < nc;
#pragma unroll
            for (int u = 0; u < B; ++u)
                v[u] = (ok && q0 + u < ns) ? __ldg(base + 128 * j + (size_t)(q0 + u) * cs) : (T)0;
        };
        load(0, 0);
        __syncthreads();
        if ((int)threadIdx.x < ns) s_sig[threadIdx.x] = dens ? (T)dens[tv.seg_panel[s0 + threadIdx.x]] : (T)1;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if ((int)threadIdx.x + 128 * j >= nc) continue;
            T a = acc[j];
            for (int q0 = 0; q0 < ns; q0 += B) {
                if (j > 0 || q0 > 0) load(j, q0);
#pragma unroll
                for (int u = 0; u < B; ++u)
                    if (q0 + u < ns) a = fma(s_sig[q0 + u], v[u], a);
            }
            acc[j] = a;
        }
    }
    T *out = M + (size_t)(tv.leaf0 + leaf) * cs;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = threadIdx.x + 128 * j;
        if (k < nc) out[k] = acc[j];
    }
}

// (leaf, panel) key of every quadrature point, and its index
__global__ void k_seg_keys(TreeView tv, const int *qpanel, uint64_t *key, int *idx) {
    const int leaf = blockIdx.x;
    for (int i = tv.qp_beg[leaf] + threadIdx.x; i < tv.qp_beg[leaf + 1]; i += blockDim.x) {
        key[i] = ((uint64_t)leaf << 32) | (uint32_t)qpanel[i];
        idx[i] = i;
    }
}

__global__ void k_seg_flags(const uint64_t *key, int64_t n, int *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// segment g = pos[i] starts at sorted point i: its first point, leaf, panel
__global__ void k_seg_write(const uint64_t *key, const int *flag, const int *pos, int64_t n, int nseg,
                            int *pt_beg, int *seg_leaf, int *seg_panel) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) {
        const int g = pos[i];
        pt_beg[g] = (int)i;
        seg_leaf[g] = (int)(key[i] >> 32);
        seg_panel[g] = (int)(uint32_t)(key[i] & 0xffffffffu);
    }
    if (i == n - 1) pt_beg[nseg] = (int)n;
}

// seg_beg[l] = the first segment of a leaf >= l (segments sorted by leaf)
__global__ void k_seg_leaf_beg(const int *seg_leaf, int nseg, int nleaf, int *seg_beg) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > nleaf) return;
    int lo = 0, hi = nseg;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (seg_leaf[mid] < l) lo = mid + 1;
        else hi = mid;
    }
    seg_beg[l] = lo;
}

template <class V>
__global__ void k_seg_gather(const V *rec, const int *idx, int64_t n, V *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = rec[idx[i]];
}

template <class T>
static bool build_p2m_moments_t(Mesh &m, Tree &t, const typename V4T<T>::t *rec, DArray<T> &mom) {
    using V4 = typename V4T<T>::t;
    cudaStream_t s = m.stream;
    const int64_t n = m.nqp;
    const int p = m.opt.p, cs = cell_stride(p);
    if ((p + 1) * (p + 1) > P2M_SEG_MAXNC || n <= 0 || n >= ((int64_t)1 << 31) || t.nleaf <= 0) return false;
    // the points' (leaf, panel) keys, sorted stably: points already come in
    // leaf order, so each leaf's points end up grouped by panel
    DArray<uint64_t> key, key_s;
    DArray<int> idx, idx_s;
    key.alloc(n);
    key_s.alloc(n);
    idx.alloc(n);
    idx_s.alloc(n);
    const TreeView tv = view(t);
    k_seg_keys<<<t.nleaf, 128, 0, s>>>(tv, m.qp_panel.p, key.p, idx.p);
    BEM_CHECK_LAUNCH();
    int lb = 1;
    while (((int64_t)1 << lb) < (int64_t)t.nleaf) ++lb;
    radix_sort_u64(key.p, idx.p, key_s.p, idx_s.p, n, 32 + lb, s);
    key.release();
    idx.release();
    DArray<int> flag, pos;
    flag.alloc(n);
    pos.alloc(n);
    k_seg_flags<<<cdiv(n, 256), 256, 0, s>>>(key_s.p, n, flag.p);
    BEM_CHECK_LAUNCH();
    scan_exclusive_i32(flag.p, pos.p, n, s);
    int last_pos = 0, last_flag = 0;
    BEM_CUDA(cudaMemcpyAsync(&last_pos, pos.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(&last_flag, flag.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    const int nseg = last_pos + last_flag;
    // the moments may take at most half of the free device memory
    const size_t bytes = (size_t)nseg * cs * sizeof(T);
    size_t fr = 0, tot = 0;
    BEM_CUDA(cudaMemGetInfo(&fr, &tot));
    if (nseg <= 0 || bytes > fr / 2) return false;
    DArray<int> pt_beg, seg_leaf;
    pt_beg.alloc((size_t)nseg + 1);
    seg_leaf.alloc(nseg);
    t.p2m_seg_panel.alloc(nseg);
    k_seg_write<<<cdiv(n, 256), 256, 0, s>>>(key_s.p, flag.p, pos.p, n, nseg, pt_beg.p, seg_leaf.p,
                                             t.p2m_seg_panel.p);
    BEM_CHECK_LAUNCH();
    t.p2m_seg_beg.alloc((size_t)t.nleaf + 1);
    k_seg_leaf_beg<<<cdiv((int64_t)t.nleaf + 1, 256), 256, 0, s>>>(seg_leaf.p, nseg, t.nleaf, t.p2m_seg_beg.p);
    BEM_CHECK_LAUNCH();
    // the points' records in segment order, then the point P2M with every
    // segment as a leaf of its own and unit density
    DArray<V4> rp;
    rp.alloc(n);
    k_seg_gather<V4><<<cdiv(n, 256), 256, 0, s>>>(rec, idx_s.p, n, rp.p);
    BEM_CHECK_LAUNCH();
    mom.alloc((size_t)nseg * cs);
    BEM_CUDA(cudaMemsetAsync(mom.p, 0, bytes, s));
    TreeView sv = tv;
    sv.qp_beg = pt_beg.p;
    sv.leaf0 = 0;
    sv.nleaf = nseg;
    const T inv_h = (T)(1.0 / (m.side / (double)(1 << t.L)));
    p2m_dispatch<T>(sv, nseg, SRC_QUAD, rp.p, nullptr, nullptr, p, cs, inv_h, mom.p, s);
    BEM_CUDA(cudaStreamSynchronize(s));  // the temporaries are released on return
    return true;
}

void build_p2m_moments(Mesh &m, Tree &t) {
    auto drop = [&]() {
        t.p2m_seg_p = -1;
        t.p2m_seg_beg.release();
        t.p2m_seg_panel.release();
        t.p2m_seg_f.release();
        t.p2m_seg_d.release();
    };
    drop();
    if ((m.opt.flags & (BEM_FLAG_P2M_FROM_POINTS | BEM_FLAG_NO_FAR)) || !t.has_qp || t.L < 2) return;
    bool ok = false;
    try {
        if (m.opt.precision == BEM_MIXED) ok = build_p2m_moments_t<float>(m, t, m.qp32.p, t.p2m_seg_f);
        else ok = build_p2m_moments_t<double>(m, t, m.qp64r.p, t.p2m_seg_d);
    } catch (const Error &e) {
        // out of device memory (or over the process's cap): P2M works from
        // the points, as with BEM_FLAG_P2M_FROM_POINTS
        if (e.code != BEM_ENOMEM) throw;
        BEM_CUDA(cudaStreamSynchronize(m.stream));
        ok = false;
    }
    if (ok) t.p2m_seg_p = m.opt.p;
    else drop();
}

template <class T>
static const T *seg_moments(const TreeView &tv);
template <>
const float *seg_moments<float>(const TreeView &tv) { return tv.seg_f; }
template <>
const double *seg_moments<double>(const TreeView &tv) { return tv.seg_d; }

template <class T>
void p2m_leaves(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src, const int *qpanel,
                const double *dens, int p, int cs, T inv_h, T *M, cudaStream_t s) {
    if (nleaf <= 0) return;
    const T *mom = seg_moments<T>(tv);
    if (sk == SRC_QUAD && tv.seg_beg && mom && tv.seg_p == p) {
        k_p2m_seg<T><<<nleaf, 128, 0, s>>>(tv, mom, dens, (p + 1) * (p + 1), cs, M);
        BEM_CHECK_LAUNCH();
        return;
    }
    p2m_dispatch<T>(tv, nleaf, sk, src, qpanel, dens, p, cs, inv_h, M, s);
}

// ------------------------------------------------------------------- L2P
// One CTA per leaf, one target per thread.  The leaf's local expansion (the
// compact real layout, (P+1)^2 values) is staged in shared memory and read
// with compile-time offsets (every lane reads the same word: a broadcast).
// With L_n^{-m} = (-1)^m conj(L_n^m) and conj(R_n^{-m}) = (-1)^m R_n^m the
// sums over m < 0 fold onto m > 0:
//   potential  phi = sum_n L_n^0 R_n^0 + 2 sum_{m>0} Re(L_n^m conj(R_n^m)),
//   gradient   L'_1^l = sum_{n,m} L_{n+1}^{m+l} conj(R_n^m) (n <= P-1), whose
//              m < 0 terms are conj(L_{n+1}^m) R_n^m (l = 0) and
//              L_{n+1}^0 R_n^1 (l = 1, m = -1), -conj(L_{n+1}^{m-1}) R_n^m (l = 1, m < -1),
// grad phi = (-Re L'_1^1, -Im L'_1^1, Re L'_1^0) / h^2, phi / h (h = cell size).
template <class T, int TGT, int P>
__global__ void __launch_bounds__(128)
k_l2p_c(TreeView tv, const typename V4T<T>::t *tgt, const typename V4T<T>::t *nrm, int cs, T inv_h, const T *L,
        T *out, ApplyEpi epi) {
    constexpr int NC = (P + 1) * (P + 1);
    constexpr bool DN = TGT == TGT_CEN_DN || TGT == TGT_QUAD_DN;
    __shared__ T sl[NC];
    const int leaf = blockIdx.x;
    const int *beg = TGT == TGT_CEN_DN ? tv.cen_beg : (TGT == TGT_CHG_PHI ? tv.chg_beg : tv.qp_beg);
    const int b = beg[leaf], e = beg[leaf + 1];
    if (b == e) return;
    const T *src = L + (size_t)(tv.leaf0 + leaf) * cs;
    for (int k = threadIdx.x; k < NC; k += blockDim.x) sl[k] = src[k];
    __syncthreads();
    auto lre = [&](int n, int m) { return sl[n * n + (m == 0 ? 0 : 2 * m - 1)]; };
    auto lim = [&](int n, int m) { return m == 0 ? (T)0 : sl[n * n + 2 * m]; };
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const typename V4T<T>::t r = tgt[i];
        const T x = r.x * inv_h, y = r.y * inv_h, z = r.z * inv_h;
        if constexpr (DN) {
            T g0r = 0, g1r = 0, g1i = 0;  // Re L'_1^0, L'_1^1
            regular_solid_c<T, P - 1>(x, y, z, [&](int n, int m, T re, T im) {
                // L_{n+1}^m conj(R) and, for m > 0, conj(L_{n+1}^m) R: together 2 Re(L conj R)
                const T ar = lre(n + 1, m), ai = lim(n + 1, m);
                if (m == 0) g0r = fma(ar, re, g0r);
                else g0r = fma((T)2 * ar, re, fma((T)2 * ai, im, g0r));
                // L_{n+1}^{m+1} conj(R)
                const T br = lre(n + 1, m + 1), bi = lim(n + 1, m + 1);
                g1r = fma(br, re, fma(bi, im, g1r));
                g1i = fma(bi, re, fma(-br, im, g1i));
                if (m == 1) {  // the m = -1 term L_{n+1}^0 conj(R_n^{-1}) = -L_{n+1}^0 R_n^1
                    const T cr = lre(n + 1, 0);
                    g1r = fma(-cr, re, g1r);
                    g1i = fma(-cr, im, g1i);
                } else if (m > 1) {  // -conj(L_{n+1}^{m-1}) R_n^m
                    const T cr = lre(n + 1, m - 1), ci = lim(n + 1, m - 1);
                    g1r = fma(-cr, re, fma(-ci, im, g1r));
                    g1i = fma(-cr, im, fma(ci, re, g1i));
                }
            });
            const typename V4T<T>::t nn = nrm[i];
            const T f = inv_h * inv_h * (-nn.x * g1r - nn.y * g1i + nn.z * g0r);
            if (epi.y) {
                const double v = (double)f + (epi.near64 ? epi.near64[i] : 0.0);
                epi.y[i] = epi.x[i] + epi.ehat * (v * (1.0 / FOUR_PI));
            } else {
                out[i] = f;
            }
        } else {
            T a = 0;
            regular_solid_c<T, P>(x, y, z, [&](int n, int m, T re, T im) {
                const T ar = lre(n, m), ai = lim(n, m);
                if (m == 0) a = fma(ar, re, a);
                else a = fma((T)2 * ar, re, fma((T)2 * ai, im, a));
            });
            out[i] = inv_h * a;
        }
    }
}

template <class T, int TGT, int P>
static void l2p_launch_c(const TreeView &tv, int nleaf, int nth, const typename V4T<T>::t *tgt,
                         const typename V4T<T>::t *nrm, int cs, T inv_h, const T *L, T *out, cudaStream_t s,
                         ApplyEpi epi) {
    k_l2p_c<T, TGT, P><<<nleaf, nth, 0, s>>>(tv, tgt, nrm, cs, inv_h, L, out, epi);
    BEM_CHECK_LAUNCH();
}

template <class T, int TGT>
static bool l2p_order(const TreeView &tv, int nleaf, int nth, int p, const typename V4T<T>::t *tgt,
                      const typename V4T<T>::t *nrm, int cs, T inv_h, const T *L, T *out, cudaStream_t s,
                      ApplyEpi epi) {
    switch (p) {
        case 6: l2p_launch_c<T, TGT, 6>(tv, nleaf, nth, tgt, nrm, cs, inv_h, L, out, s, epi); return true;
        case 8: l2p_launch_c<T, TGT, 8>(tv, nleaf, nth, tgt, nrm, cs, inv_h, L, out, s, epi); return true;
        case 10: l2p_launch_c<T, TGT, 10>(tv, nleaf, nth, tgt, nrm, cs, inv_h, L, out, s, epi); return true;
        case 12: l2p_launch_c<T, TGT, 12>(tv, nleaf, nth, tgt, nrm, cs, inv_h, L, out, s, epi); return true;
        default: return false;
    }
}

template <class T>
bool l2p_leaves_c(const TreeView &tv, int nleaf, int nth, TgtKind tk, int p, const typename V4T<T>::t *tgt,
                  const typename V4T<T>::t *nrm, int cs, T inv_h, const T *L, T *out, cudaStream_t s,
                  ApplyEpi epi) {
    if (epi.y && tk != TGT_CEN_DN) throw Error(BEM_EUNSUPPORTED, "L2P epilogue: collocation targets only");
    if (nleaf <= 0) return true;
    switch (tk) {
        case TGT_CEN_DN: return l2p_order<T, TGT_CEN_DN>(tv, nleaf, nth, p, tgt, nrm, cs, inv_h, L, out, s, epi);
        case TGT_QUAD_DN: return l2p_order<T, TGT_QUAD_DN>(tv, nleaf, nth, p, tgt, nrm, cs, inv_h, L, out, s, epi);
        case TGT_CHG_PHI: return l2p_order<T, TGT_CHG_PHI>(tv, nleaf, nth, p, tgt, nrm, cs, inv_h, L, out, s, epi);
        case TGT_QUAD_PHI: return l2p_order<T, TGT_QUAD_PHI>(tv, nleaf, nth, p, tgt, nrm, cs, inv_h, L, out, s, epi);
    }
    return false;
}

template bool l2p_leaves_c<float>(const TreeView &, int, int, TgtKind, int, const float4 *, const float4 *, int,
                                  float, const float *, float *, cudaStream_t, ApplyEpi);
template bool l2p_leaves_c<double>(const TreeView &, int, int, TgtKind, int, const double4 *, const double4 *, int,
                                   double, const double *, double *, cudaStream_t, ApplyEpi);

template void p2m_leaves<float>(const TreeView &, int, SrcKind, const float4 *, const int *, const double *, int,
                                int, float, float *, cudaStream_t);
template void p2m_leaves<double>(const TreeView &, int, SrcKind, const double4 *, const int *, const double *, int,
                                 int, double, double *, cudaStream_t);
}  // namespace bem
