// Direct (all-pairs) products between the point charges and the surface:
// (B q)_i at the collocation points and (C s)_k at the charges.
//
// For the sizes where n_c * n_p * quad_points is modest (every molecule in
// the single-molecule and batched workloads) the direct sum is both cheaper
// and exact to rounding, while the fast multipole pass over a
// one-cell-separated octree has a worst case (a charge at a cell corner)
// whose truncation error converges only like (sqrt(3)/2)^p.  Large systems
// (many molecules) use the fast multipole pass; opt.charge_mode selects.
//
// Coordinates are taken relative to the root-cube centre; in FP32 each one is
// carried as a pair hi + lo (hi = the FP32 rounding, lo = the FP32 rounding of
// the rest) and a difference is formed as (hi_t - hi_s) + (lo_t - lo_s): the
// first term is exact for nearby points, so a pair's difference keeps about
// 2^-24 of its own length instead of 2^-24 of the distance from the centre
// (charges a few hundredths of an A from a quadrature or collocation point).
// Each thread sums one tile in a short accumulator and adds the tile total
// to a second one, and the partial sums of the source splits are reduced in
// FP64.
#include "bem_internal.cuh"

namespace bem {

namespace {
template <class T> struct V4D;
template <> struct V4D<float> { using t = float4; };
template <> struct V4D<double> { using t = double4; };
__device__ __forceinline__ float rsqd(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqd(double x) { return rsqrt(x); }
}  // namespace

constexpr int DIRECT_THREADS = 256;

template <class T, int SRC, int TGT>
__global__ void __launch_bounds__(DIRECT_THREADS)
k_direct(int64_t ntgt, int64_t nsrc, int64_t chunk, const double *tpos, const double *tnrm,
         const double *spos, const double *sw, const int *qpanel, const double *dens, double ox,
         double oy, double oz, T *part) {
    using V4 = typename V4D<T>::t;
    constexpr bool SPLIT = sizeof(T) == 4;  // coordinates as hi + lo pairs
    __shared__ V4 sh[DIRECT_THREADS];
    __shared__ float4 shl[SPLIT ? DIRECT_THREADS : 1];
    const int64_t i = blockIdx.x * (int64_t)DIRECT_THREADS + threadIdx.x;
    const int64_t sb = (int64_t)blockIdx.y * chunk;
    const int64_t se = min(nsrc, sb + chunk);
    constexpr bool DN = TGT == TGT_CEN_DN || TGT == TGT_QUAD_DN;  // normal field, else potential
    T cx = 0, cy = 0, cz = 0, nx = 0, ny = 0, nz = 0;
    float lx = 0.f, ly = 0.f, lz = 0.f;
    if (i < ntgt) {
        const double px = tpos[3 * i] - ox, py = tpos[3 * i + 1] - oy, pz = tpos[3 * i + 2] - oz;
        cx = (T)px;
        cy = (T)py;
        cz = (T)pz;
        if (SPLIT) {
            lx = (float)(px - (double)cx);
            ly = (float)(py - (double)cy);
            lz = (float)(pz - (double)cz);
        }
        if (DN) {
            nx = (T)tnrm[3 * i];
            ny = (T)tnrm[3 * i + 1];
            nz = (T)tnrm[3 * i + 2];
        }
    }
    T outer = 0;
    for (int64_t b = sb; b < se; b += DIRECT_THREADS) {
        __syncthreads();
        const int64_t k = b + threadIdx.x;
        V4 r;
        r.x = r.y = r.z = r.w = 0;
        float4 rl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < se) {
            const double px = spos[3 * k] - ox, py = spos[3 * k + 1] - oy, pz = spos[3 * k + 2] - oz;
            r.x = (T)px;
            r.y = (T)py;
            r.z = (T)pz;
            if (SPLIT) rl = make_float4((float)(px - (double)r.x), (float)(py - (double)r.y), (float)(pz - (double)r.z), 0.f);
            double w;
            if (SRC == SRC_QUAD) w = sw[k] * dens[qpanel[k]];
            else w = dens ? dens[k] : sw[k];
            r.w = (T)w;
        }
        sh[threadIdx.x] = r;
        if (SPLIT) shl[threadIdx.x] = rl;
        __syncthreads();
        const int cnt = (int)min((int64_t)DIRECT_THREADS, se - b);
        T acc = 0;
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
            const V4 y = sh[j];
            T dx = cx - y.x, dy = cy - y.y, dz = cz - y.z;
            if (SPLIT) {
                const float4 yl = shl[j];
                dx += (T)(lx - yl.x);
                dy += (T)(ly - yl.y);
                dz += (T)(lz - yl.z);
            }
            const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const T ri = rsqd(r2);
            if (DN) {
                const T nd = fma(nx, dx, fma(ny, dy, nz * dz));
                acc = fma(y.w * nd, ri * ri * ri, acc);
            } else {
                acc = fma(y.w, ri, acc);
            }
        }
        outer += acc;
    }
    if (i < ntgt) part[(size_t)blockIdx.y * ntgt + i] = DN ? -outer : outer;
}

template <class T>
__global__ void k_direct_reduce(const T *part, int nsplit, int64_t n, double scale, double *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += (double)part[(size_t)k * n + i];
    out[i] = scale * s;
}

// out_j = sum_q (qw_jq / A_j) v_jq: the rule's average over panel j
__global__ void k_panel_avg(const double *v, const int *qp_of_panel, const double *qw, const double *area,
                            int nq, int64_t np, double *out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double a = 0.0;
    for (int q = 0; q < nq; ++q) {
        const int k = qp_of_panel[j * nq + q];
        a += qw[k] * v[k];
    }
    out[j] = a / area[j];
}

template <class T>
static void direct_impl(Mesh &m, SrcKind sk, TgtKind tk, const double *dens, double *out,
                        DArray<T> &part) {
    cudaStream_t s = m.stream;
    const int64_t ntgt = (tk == TGT_CEN_DN) ? m.np : ((tk == TGT_QUAD_DN || tk == TGT_QUAD_PHI) ? m.nqp : m.nc);
    // Galerkin rows: the values at the quadrature points, then the rule's
    // average over each panel
    double *const final_out = out;
    if (tk == TGT_QUAD_DN) {
        if (!m.nrmq64.p || m.gq_tmp.n < (size_t)m.nqp) throw Error(BEM_EUNSUPPORTED, "Galerkin geometry not built");
        out = m.gq_tmp.p;
    }
    const int64_t nsrc = (sk == SRC_QUAD) ? m.nqp : m.nc;
    if (ntgt == 0) return;
    if (nsrc == 0) {
        BEM_CUDA(cudaMemsetAsync(final_out, 0, (tk == TGT_QUAD_DN ? m.np : ntgt) * sizeof(double), s));
        return;
    }
    const int tblocks = cdiv(ntgt, DIRECT_THREADS);
    // enough CTAs to fill the GPU about twice (16 per SM), splits of at least 512 sources
    int nsplit = std::max(1, (int)std::min<int64_t>(cdiv(nsrc, 512), std::max(1, 2432 / tblocks)));
    nsplit = std::min(nsplit, 65535);
    int64_t chunk = (nsrc + nsplit - 1) / nsplit;
    chunk = ((chunk + DIRECT_THREADS - 1) / DIRECT_THREADS) * DIRECT_THREADS;
    nsplit = (int)((nsrc + chunk - 1) / chunk);
    const size_t need = (size_t)nsplit * ntgt;
    if (part.n < need) part.alloc(need);
    const double ox = m.root_min[0] + 0.5 * m.side, oy = m.root_min[1] + 0.5 * m.side,
                 oz = m.root_min[2] + 0.5 * m.side;
    const double *tpos = (tk == TGT_CEN_DN) ? m.cen64.p : ((tk == TGT_QUAD_DN || tk == TGT_QUAD_PHI) ? m.qpg64.p : m.chgg64.p);
    const double *spos = (sk == SRC_QUAD) ? m.qpg64.p : m.chgg64.p;
    const double *sw = (sk == SRC_QUAD) ? m.qw64.p : m.q64.p;
    dim3 grid(tblocks, nsplit);
    if (sk == SRC_QUAD && tk == TGT_CHG_PHI)
        k_direct<T, SRC_QUAD, TGT_CHG_PHI><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, nullptr, spos, sw, m.qp_panel.p, dens, ox, oy, oz, part.p);
    else if (sk == SRC_CHARGE && tk == TGT_CEN_DN)
        k_direct<T, SRC_CHARGE, TGT_CEN_DN><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, m.nrm64.p, spos, sw, nullptr, dens, ox, oy, oz, part.p);
    else if (sk == SRC_QUAD && tk == TGT_CEN_DN)
        k_direct<T, SRC_QUAD, TGT_CEN_DN><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, m.nrm64.p, spos, sw, m.qp_panel.p, dens, ox, oy, oz, part.p);
    else if (sk == SRC_CHARGE && tk == TGT_QUAD_DN)
        k_direct<T, SRC_CHARGE, TGT_QUAD_DN><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, m.nrmq64.p, spos, sw, nullptr, dens, ox, oy, oz, part.p);
    else if (sk == SRC_CHARGE && tk == TGT_QUAD_PHI)
        k_direct<T, SRC_CHARGE, TGT_QUAD_PHI><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, nullptr, spos, sw, nullptr, dens, ox, oy, oz, part.p);
    else if (sk == SRC_QUAD && (tk == TGT_QUAD_DN || tk == TGT_QUAD_PHI))
        throw Error(BEM_EUNSUPPORTED, "direct quadrature-to-quadrature sums not built");
    else
        k_direct<T, SRC_CHARGE, TGT_CHG_PHI><<<grid, DIRECT_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, nullptr, spos, sw, nullptr, dens, ox, oy, oz, part.p);
    BEM_CHECK_LAUNCH();
    k_direct_reduce<T><<<cdiv(ntgt, 256), 256, 0, s>>>(part.p, nsplit, ntgt, 1.0 / FOUR_PI, out);
    BEM_CHECK_LAUNCH();
    if (tk == TGT_QUAD_DN) {
        k_panel_avg<<<cdiv(m.np, 256), 256, 0, s>>>(out, m.qp_of_panel.p, m.qw64.p, m.area64.p, (int)m.nq,
                                                    m.np, final_out);
        BEM_CHECK_LAUNCH();
    }
}

// out_j = sum_q qw_jq v_jq (the rule's weights include the panel area)
__global__ void k_panel_wsum(const double *v, const int *qp_of_panel, const double *qw, int nq, int64_t np,
                             double *out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double a = 0.0;
    for (int q = 0; q < nq; ++q) {
        const int k = qp_of_panel[j * nq + q];
        a += qw[k] * v[k];
    }
    out[j] = a;
}

// C^T q in the sorted panel order: (C^T q)_j = sum_q A_j w_q psi(y_jq) with
// psi(y) = sum_k q_k G(x_k, y), so that q . (C sigma) = (C^T q) . sigma and
// the solvation energy of any sigma is one dot product (Eq. energy).  Built
// in the product's precision for meshes whose charge sums are direct.
void build_ctq(Mesh &m) {
    m.ctq_ok = false;
    if (m.nc == 0 || !charge_direct(m)) return;
    if (m.ctq.n < (size_t)m.np) m.ctq.alloc(m.np);
    DArray<double> psi;
    psi.alloc(m.nqp);
    direct_pass(m, SRC_CHARGE, TGT_QUAD_PHI, nullptr, psi.p);
    k_panel_wsum<<<cdiv(m.np, 256), 256, 0, m.stream>>>(psi.p, m.qp_of_panel.p, m.qw64.p, (int)m.nq, m.np, m.ctq.p);
    BEM_CHECK_LAUNCH();
    charge_near_ct(m, m.q64.p, m.ctq.p);
    BEM_CUDA(cudaStreamSynchronize(m.stream));
    m.ctq_ok = true;
}

void direct_pass(Mesh &m, SrcKind sk, TgtKind tk, const double *dens, double *out) {
    if (m.opt.precision == BEM_MIXED) direct_impl<float>(m, sk, tk, dens, out, m.dpart_f);
    else direct_impl<double>(m, sk, tk, dens, out, m.dpart_d);
}

bool charge_direct(const Mesh &m) {
    if (m.opt.charge_mode == BEM_CHARGE_DIRECT) return true;
    if (m.opt.charge_mode == BEM_CHARGE_FMM) return false;
    return (double)m.nc * (double)m.nqp <= 4e10;
}

void charge_pass(Mesh &m, SrcKind sk, TgtKind tk, const double *dens, double *out) {
    if (charge_direct(m)) direct_pass(m, sk, tk, dens, out);
    else fmm_pass(m, m.tc, sk, tk, dens, out, false);
}

}  // namespace bem
