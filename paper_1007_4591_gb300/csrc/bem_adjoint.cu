// Transposed operator and adjoint gradients of the solvation energy.
//
// dG(q, x) = kappa/(2 eps_in) q^T C(x) sigma,  (I + Ehat K') sigma = -Ehat B(x) q,
// kappa = 4 pi 332.0637 (the matrix form of Sec. 2.1; the mesh, hence K', does
// not depend on the charges).  With lam solving A^T lam = C^T q:
//   d dG / d q_k = kappa/(2 eps_in) [ (C sigma)_k - Ehat (B^T lam)_k ]
//   d dG / d x_k = kappa/(2 eps_in) q_k [ grad_x (C sigma)_k - Ehat sum_i lam_i grad_{x_k} B_ik ].
// B^T lam at x is the potential of dipoles lam_i n_i placed at the collocation
// points, and sum_i lam_i grad_{x_k} B_ik its gradient; C^T q is the
// potential of the charges at the quadrature points summed over each panel.
// The products between charges and surface are direct sums here; K'^T is a
// fast multipole pass (fmm_pass_t) plus the transposed near-singular table.
// In the Galerkin form K' and B are K'_G and B_G (every row averaged over its
// panel by the rule): their transposes place the dipoles lam_i w_q n_i at the
// quadrature points of panel i instead of lam_i n_i at its centroid.
#include <algorithm>

#include "bem_internal.cuh"

namespace bem {

int gmres_solve(Mesh &m, const double *b, double *x, bool transpose, bem_solve_stats *st);

namespace {
template <class T> struct V4A;
template <> struct V4A<float> { using t = float4; };
template <> struct V4A<double> { using t = double4; };
__device__ __forceinline__ float rsqa(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqa(double x) { return rsqrt(x); }
}  // namespace

enum AdjSrc { AS_QUAD = 0, AS_CHARGE = 1, AS_DIPOLE = 2 };
enum AdjTgt { AT_CHG_GRAD = 0, AT_QUAD_PHI = 1 };
constexpr int ADJ_THREADS = 256;

// Direct sums of G = 1/(4 pi r) and its gradient (the 1/(4 pi) is applied in
// the reduction).  Monopole s at y: phi = s/r, grad = -s d/r^3 (d = x - y).
// Dipole p at c: phi = p.d/r^3, grad = p/r^3 - 3 (p.d) d/r^5.
template <class T, int SK, int TK>
__global__ void __launch_bounds__(ADJ_THREADS)
k_direct_adj(int64_t ntgt, int64_t nsrc, int64_t chunk, const double *tpos, const double *spos,
             const double *sw, const double *snrm, const int *qpanel, const double *dens, double ox,
             double oy, double oz, T *part) {
    using V4 = typename V4A<T>::t;
    // FP32: coordinates as hi + lo pairs, differences (hi - hi) + (lo - lo)
    // (exact first term for nearby points; see k_direct)
    constexpr bool SPLIT = sizeof(T) == 4;
    __shared__ V4 sa[ADJ_THREADS], sb[ADJ_THREADS];
    __shared__ float4 sl[SPLIT ? ADJ_THREADS : 1];
    const int64_t i = blockIdx.x * (int64_t)ADJ_THREADS + threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * chunk, s1 = min(nsrc, s0 + chunk);
    T x = 0, y = 0, z = 0;
    float lx = 0.f, ly = 0.f, lz = 0.f;
    if (i < ntgt) {
        const double px = tpos[3 * i] - ox, py = tpos[3 * i + 1] - oy, pz = tpos[3 * i + 2] - oz;
        x = (T)px;
        y = (T)py;
        z = (T)pz;
        if (SPLIT) {
            lx = (float)(px - (double)x);
            ly = (float)(py - (double)y);
            lz = (float)(pz - (double)z);
        }
    }
    T o0 = 0, o1 = 0, o2 = 0, o3 = 0;
    for (int64_t b = s0; b < s1; b += ADJ_THREADS) {
        __syncthreads();
        const int64_t k = b + threadIdx.x;
        V4 a, c;
        a.x = a.y = a.z = a.w = 0;
        c.x = c.y = c.z = c.w = 0;
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < s1) {
            const double px = spos[3 * k] - ox, py = spos[3 * k + 1] - oy, pz = spos[3 * k + 2] - oz;
            a.x = (T)px;
            a.y = (T)py;
            a.z = (T)pz;
            if (SPLIT) al = make_float4((float)(px - (double)a.x), (float)(py - (double)a.y), (float)(pz - (double)a.z), 0.f);
            if (SK == AS_QUAD) a.w = (T)(sw[k] * dens[qpanel[k]]);
            else if (SK == AS_CHARGE) a.w = (T)sw[k];
            else {
                const double l = dens[k];
                c.x = (T)(l * snrm[3 * k]);
                c.y = (T)(l * snrm[3 * k + 1]);
                c.z = (T)(l * snrm[3 * k + 2]);
            }
        }
        sa[threadIdx.x] = a;
        sb[threadIdx.x] = c;
        if (SPLIT) sl[threadIdx.x] = al;
        __syncthreads();
        const int cnt = (int)min((int64_t)ADJ_THREADS, s1 - b);
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int j = 0; j < cnt; ++j) {
            const V4 sp = sa[j];
            T dx = x - sp.x, dy = y - sp.y, dz = z - sp.z;
            if (SPLIT) {
                const float4 q = sl[j];
                dx += (T)(lx - q.x);
                dy += (T)(ly - q.y);
                dz += (T)(lz - q.z);
            }
            const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (r2 == (T)0) continue;  // a dummy slot or a coincident point
            const T ri = rsqa(r2), ri3 = ri * ri * ri;
            if (SK != AS_DIPOLE) {
                a0 = fma(sp.w, ri, a0);
                if (TK == AT_CHG_GRAD) {
                    const T f = -sp.w * ri3;
                    a1 = fma(f, dx, a1);
                    a2 = fma(f, dy, a2);
                    a3 = fma(f, dz, a3);
                }
            } else {
                const V4 pm = sb[j];
                const T pd = fma(pm.x, dx, fma(pm.y, dy, pm.z * dz));
                a0 = fma(pd, ri3, a0);
                if (TK == AT_CHG_GRAD) {
                    const T f = (T)3 * pd * ri3 * ri * ri;
                    a1 += pm.x * ri3 - f * dx;
                    a2 += pm.y * ri3 - f * dy;
                    a3 += pm.z * ri3 - f * dz;
                }
            }
        }
        o0 += a0;
        o1 += a1;
        o2 += a2;
        o3 += a3;
    }
    if (i < ntgt) {
        T *pp = part + ((size_t)blockIdx.y * ntgt + i) * 4;
        pp[0] = o0;
        pp[1] = o1;
        pp[2] = o2;
        pp[3] = o3;
    }
}

template <class T>
__global__ void k_reduce4(const T *part, int nsplit, int64_t n, double scale, double *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[4] = {0, 0, 0, 0};
    for (int k = 0; k < nsplit; ++k)
        for (int c = 0; c < 4; ++c) a[c] += (double)part[((size_t)k * n + i) * 4 + c];
    for (int c = 0; c < 4; ++c) out[i * 4 + c] = scale * a[c];
}

// out[ntgt][4] = (phi, grad phi) / (4 pi) (grad entries zero for AT_QUAD_PHI)
template <class T>
static void direct_adj(Mesh &m, AdjSrc sk, AdjTgt tk, const double *dens, double *out) {
    cudaStream_t s = m.stream;
    const int64_t ntgt = (tk == AT_CHG_GRAD) ? m.nc : m.nqp;
    // Galerkin: the dipoles of B_G^T sit at every quadrature point, their
    // moments lam_j w_q in m.lamq (galerkin_moments)
    const bool gq = sk == AS_DIPOLE && m.opt.galerkin;
    const int64_t nsrc = (sk == AS_QUAD) ? m.nqp : (sk == AS_CHARGE ? m.nc : (gq ? m.nqp : m.np));
    if (ntgt == 0) return;
    if (nsrc == 0) {
        BEM_CUDA(cudaMemsetAsync(out, 0, ntgt * 4 * sizeof(double), s));
        return;
    }
    const int tblocks = cdiv(ntgt, ADJ_THREADS);
    int nsplit = std::max(1, (int)std::min<int64_t>(cdiv(nsrc, 4096), std::max(1, 1216 / tblocks)));
    nsplit = std::min(nsplit, 65535);
    int64_t chunk = (nsrc + nsplit - 1) / nsplit;
    chunk = ((chunk + ADJ_THREADS - 1) / ADJ_THREADS) * ADJ_THREADS;
    nsplit = (int)((nsrc + chunk - 1) / chunk);
    DArray<T> part;
    part.alloc((size_t)nsplit * ntgt * 4);
    const double ox = m.root_min[0] + 0.5 * m.side, oy = m.root_min[1] + 0.5 * m.side,
                 oz = m.root_min[2] + 0.5 * m.side;
    const double *tpos = (tk == AT_CHG_GRAD) ? m.chgg64.p : m.qpg64.p;
    dim3 grid(tblocks, nsplit);
    if (sk == AS_QUAD && tk == AT_CHG_GRAD)
        k_direct_adj<T, AS_QUAD, AT_CHG_GRAD><<<grid, ADJ_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, m.qpg64.p, m.qw64.p, nullptr, m.qp_panel.p, dens, ox, oy, oz, part.p);
    else if (sk == AS_DIPOLE && tk == AT_CHG_GRAD)
        k_direct_adj<T, AS_DIPOLE, AT_CHG_GRAD><<<grid, ADJ_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, gq ? m.qpg64.p : m.cen64.p, nullptr, gq ? m.nrmq64.p : m.nrm64.p, nullptr,
            gq ? m.lamq.p : dens, ox, oy, oz, part.p);
    else if (sk == AS_CHARGE && tk == AT_QUAD_PHI)
        k_direct_adj<T, AS_CHARGE, AT_QUAD_PHI><<<grid, ADJ_THREADS, 0, s>>>(
            ntgt, nsrc, chunk, tpos, m.chgg64.p, m.q64.p, nullptr, nullptr, nullptr, ox, oy, oz, part.p);
    else
        throw Error(BEM_EUNSUPPORTED, "direct adjoint combination not built");
    BEM_CHECK_LAUNCH();
    k_reduce4<T><<<cdiv(ntgt, 256), 256, 0, s>>>(part.p, nsplit, ntgt, 1.0 / FOUR_PI, out);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));  // `part` is released on return
}

static void direct_adjoint(Mesh &m, AdjSrc sk, AdjTgt tk, const double *dens, double *out) {
    if (m.opt.precision == BEM_MIXED) direct_adj<float>(m, sk, tk, dens, out);
    else direct_adj<double>(m, sk, tk, dens, out);
}

// y = A^T x = x + Ehat (K'^T x)
// four lanes per row, as k_apply_A
__global__ void k_apply_At(const double *x, const double *ktx, const int *off, const int *col,
                           const double *val, double ehat, int64_t n, double *y) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2;
    const int sub = threadIdx.x & 3;
    double k = 0.0;
    if (i < n && off)
        for (int e = off[i] + sub; e < off[i + 1]; e += 4) k += val[e] * x[col[e]];
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    if (i < n && sub == 0) y[i] = x[i] + ehat * (ktx[i] + k);
}

void matvec_t_sorted(Mesh &m, const double *xs, double *ys) {
    const bool nt = m.nt_nnz > 0 && !(m.opt.flags & (BEM_FLAG_NO_NEARTAB | BEM_FLAG_NO_NEAR));
    if (nt) transpose_near_table(m);
    fmm_pass_t(m, xs, m.zs.p);
    k_apply_At<<<cdiv(4 * m.np, 256), 256, 0, m.stream>>>(xs, m.zs.p, nt ? m.ntT_off.p : nullptr,
                                                       m.ntT_col.p, m.ntT_val.p, m.ehat, m.np, ys);
    BEM_CHECK_LAUNCH();
}

// per-panel sum of quadrature-point values: out_j = sum_q A_j w_q v4[k].x
__global__ void k_panel_sum4(const double *v4, const int *qop, const double *qw, int nq, int64_t np,
                             double *out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double a = 0.0;
    for (int q = 0; q < nq; ++q) {
        const int k = qop[j * nq + q];
        a += qw[k] * v4[(size_t)k * 4];
    }
    out[j] = a;
}

__global__ void k_gradients(const double *cs4, const double *bl4, const double *q, double ehat,
                            double pref, int64_t nc, double *dq, double *dx) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    dq[k] = pref * (cs4[4 * k] - ehat * bl4[4 * k]);
    for (int c = 0; c < 3; ++c) dx[3 * k + c] = pref * q[k] * (cs4[4 * k + 1 + c] - ehat * bl4[4 * k + 1 + c]);
}

void build_qp_of_panel(Mesh &m);

void adjoint_gradients(Mesh &m, double grad_out, double *dq_s, double *dx_s) {
    cudaStream_t s = m.stream;
    build_qp_of_panel(m);
    const int64_t np = m.np, nc = m.nc;
    DArray<double> cs4, bl4, ct4, rhs, lam;
    cs4.alloc((size_t)nc * 4);
    bl4.alloc((size_t)nc * 4);
    ct4.alloc((size_t)m.nqp * 4);
    rhs.alloc(np);
    lam.alloc(np);
    // C sigma and its gradient at the charges
    direct_adjoint(m, AS_QUAD, AT_CHG_GRAD, m.sigma_s.p, cs4.p);
    charge_near_phi(m, m.sigma_s.p, cs4.p, 4, 4);
    // C^T q: potential of the charges at the quadrature points, summed per panel
    direct_adjoint(m, AS_CHARGE, AT_QUAD_PHI, nullptr, ct4.p);
    k_panel_sum4<<<cdiv(np, 256), 256, 0, s>>>(ct4.p, m.qp_of_panel.p, m.qw64.p, (int)m.nq, np, rhs.p);
    BEM_CHECK_LAUNCH();
    charge_near_ct(m, m.q64.p, rhs.p);
    // A^T lam = C^T q
    BEM_CUDA(cudaMemsetAsync(lam.p, 0, np * sizeof(double), s));
    bem_solve_stats st{};
    gmres_solve(m, rhs.p, lam.p, true, &st);
    // B^T lam and its gradient: dipoles lam_i n_i at the collocation points
    // (Galerkin: lam_i w_q n_i at the quadrature points)
    if (m.opt.galerkin) galerkin_moments(m, lam.p);
    direct_adjoint(m, AS_DIPOLE, AT_CHG_GRAD, lam.p, bl4.p);
    const double pref = grad_out * FOUR_PI * KCAL / (2.0 * m.eps_in);
    k_gradients<<<cdiv(nc, 256), 256, 0, s>>>(cs4.p, bl4.p, m.q64.p, m.ehat, pref, nc, dq_s, dx_s);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bem
