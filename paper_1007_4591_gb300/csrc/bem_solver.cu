// BEM operator, restarted GMRES and energy reductions (Sec. 2.1, Sec. 2.2).
//
// All vectors here are FP64 and in the sorted panel order; the public entry
// points gather/scatter at the boundary.  GMRES (Saad & Schultz) runs on the
// device: classical Gram-Schmidt applied twice (CGS2) for the Arnoldi step,
// Givens rotations for the least-squares update, one 8-byte residual read by
// the host per iteration to decide convergence.
#include <cmath>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ permutations
__global__ void k_gather(const double *src, const int *perm, double *dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}
__global__ void k_scatter(const double *src, const int *perm, double *dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[perm[i]] = src[i];
}
__global__ void k_scatter3(const double *src, const int *perm, double *dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    dst[3 * j] = src[3 * i];
    dst[3 * j + 1] = src[3 * i + 1];
    dst[3 * j + 2] = src[3 * i + 2];
}

void gather_f64(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s) {
    k_gather<<<cdiv(n, 256), 256, 0, s>>>(src, perm, dst, n);
    BEM_CHECK_LAUNCH();
}
void scatter_f64(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s) {
    k_scatter<<<cdiv(n, 256), 256, 0, s>>>(src, perm, dst, n);
    BEM_CHECK_LAUNCH();
}
void scatter_rows3(const double *src, const int *perm, double *dst, int64_t n, cudaStream_t s) {
    k_scatter3<<<cdiv(n, 256), 256, 0, s>>>(src, perm, dst, n);
    BEM_CHECK_LAUNCH();
}

// --------------------------------------------------------------- operator
// y = x + Ehat (K'x): kx holds the fast multipole K' x (sorted order); the
// FP64 near-singular table replaces the FP32 near-field values of the pairs
// it lists.
// y = x + Ehat (K'x + table x): four lanes per row share the row's table
// entries (a dozen or so gathers each row), then add up by shuffles.
__global__ void k_apply_A(const double *x, const double *kx, const int *nt_off, const int *nt_col,
                          const double *nt_val, double ehat, int64_t n, double *y) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2;
    const int sub = threadIdx.x & 3;
    double k = 0.0;
    if (i < n && nt_off)
        for (int e = nt_off[i] + sub; e < nt_off[i + 1]; e += 4) k += nt_val[e] * x[nt_col[e]];
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    if (i < n && sub == 0) y[i] = x[i] + ehat * (kx[i] + k);
}

static void matvec_launch(Mesh &m, const double *xs, double *ys) {
    if (!m.opt.galerkin) {
        kprime_apply(m, xs, ys);  // the pass ends in the epilogue itself
    } else {
        const bool nt = m.nt_nnz > 0 && !(m.opt.flags & (BEM_FLAG_NO_NEARTAB | BEM_FLAG_NO_NEAR));
        fmm_pass(m, m.tp, SRC_QUAD, TGT_QUAD_DN, xs, m.zs.p, true);
        k_apply_A<<<cdiv(4 * m.np, 256), 256, 0, m.stream>>>(xs, m.zs.p, nt ? m.nt_off.p : nullptr,
                                                          m.nt_col.p, m.nt_val.p, m.ehat, m.np, ys);
        BEM_CHECK_LAUNCH();
    }
    if (m.tm.on) BEM_CUDA(cudaEventRecord(m.tm.ev[7], m.stream));
}

// The K' product is a fixed sequence of ~20 kernels and memsets; with
// opt.graph it is captured once (on the buffers gx -> gy, after one ordinary
// run has set every kernel attribute) and replayed as a single graph launch.
static cudaError_t set_node_priorities(cudaGraph_t g) {
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    size_t n = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n > 0) e = cudaGraphGetNodes(g, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
        cudaGraphNodeType ty;
        e = cudaGraphNodeGetType(nodes[i], &ty);
        if (e != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
        if (e != cudaSuccess) break;
        cudaLaunchAttributeValue v{};
        v.priority = is_near_field_kernel(kp.func) ? prio_lo : prio_hi;
        e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaLaunchAttributePriority, &v);
    }
    return e;
}

void matvec_sorted(Mesh &m, const double *xs, double *ys) {
    if (!m.opt.graph || m.tm.on) {
        matvec_launch(m, xs, ys);
        return;
    }
    if (!m.g_mv) {
        if (m.gx.n < (size_t)m.np) {
            m.gx.alloc(m.np);
            m.gy.alloc(m.np);
        }
        matvec_launch(m, xs, ys);  // warm-up outside the capture
        cudaGraph_t g = nullptr;
        BEM_CUDA(cudaStreamBeginCapture(m.stream, cudaStreamCaptureModeThreadLocal));
        m.capturing = true;
        try {
            matvec_launch(m, m.gx.p, m.gy.p);
        } catch (...) {
            m.capturing = false;
            cudaStreamEndCapture(m.stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        m.capturing = false;
        BEM_CUDA(cudaStreamEndCapture(m.stream, &g));
        // Kernel nodes do not keep their capturing stream's priority: give the
        // near-field kernels the lowest and every other kernel the highest, so
        // that the graph runs the two branches as the streams would.
        cudaError_t e = set_node_priorities(g);
        if (e == cudaSuccess) e = cudaGraphInstantiateWithFlags(&m.g_mv, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        BEM_CUDA(e);
        return;
    }
    if (xs != m.gx.p)
        BEM_CUDA(cudaMemcpyAsync(m.gx.p, xs, m.np * sizeof(double), cudaMemcpyDeviceToDevice, m.stream));
    BEM_CUDA(cudaGraphLaunch(m.g_mv, m.stream));
    if (ys != m.gy.p)
        BEM_CUDA(cudaMemcpyAsync(ys, m.gy.p, m.np * sizeof(double), cudaMemcpyDeviceToDevice, m.stream));
}

// --------------------------------------------------------------- BLAS-1
__global__ void k_dot_parts(const double *V, size_t ld, const double *w, int64_t n, int chunk,
                            double *part) {
    const int i = blockIdx.y, c = blockIdx.x;
    const int64_t b = (int64_t)c * chunk, e = min(n, b + chunk);
    const double *v = V + (size_t)i * ld;
    double s = 0.0;
    for (int64_t r = b + threadIdx.x; r < e; r += blockDim.x) s += v[r] * w[r];
    s = block_sum(s);
    if (threadIdx.x == 0) part[(size_t)i * gridDim.x + c] = s;
}

// out[i] (+)= sum of the parts of vector i; mode 0: store, 1: add, 2: store sqrt
__global__ void k_finish(const double *part, int nchunk, double *out, int mode) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x) s += part[(size_t)i * nchunk + c];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        if (mode == 0) out[i] = s;
        else if (mode == 1) out[i] += s;
        else out[i] = sqrt(s);
    }
}

// w -= sum_i h[i] V_i   (sign = -1)   or   w += sum_i h[i] V_i (sign = +1)
__global__ void k_multi_axpy(const double *V, size_t ld, int nvec, const double *h, double sign,
                             double *w, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double a = 0.0;
    for (int i = 0; i < nvec; ++i) a += h[i] * V[(size_t)i * ld + r];
    w[r] += sign * a;
}

__global__ void k_scale_by(double *w, const double *sc, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) w[r] *= sc[0];
}

__global__ void k_scale_by_inv(double *w, const double *d, int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) w[r] /= d[0];
}

__global__ void k_axpby(double a, const double *x, double b, const double *y, double *out,
                        int64_t n) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = a * x[r] + b * y[r];
}

// Givens update of Hessenberg column j (column-major, leading dimension m1).
__global__ void k_givens(double *H, int m1, const double *hcol, int j, double *cs, double *sn,
                         double *g, double inv_bnorm, double *out /* [0]=resid, [1]=1/norm */) {
    double *h = H + (size_t)j * m1;
    for (int i = 0; i <= j + 1; ++i) h[i] = hcol[i];
    const double wn = h[j + 1];
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double den = hypot(h[j], h[j + 1]);
    if (den > 0.0) {
        cs[j] = h[j] / den;
        sn[j] = h[j + 1] / den;
    } else {
        cs[j] = 1.0;
        sn[j] = 0.0;
    }
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    out[0] = fabs(g[j + 1]) * inv_bnorm;
    out[1] = (wn > 0.0) ? 1.0 / wn : 0.0;
}

// Back substitution  H[:k,:k] y = g[:k].
__global__ void k_backsolve(const double *H, int m1, const double *g, int k, double *y) {
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * m1 + i] * y[l];
        const double d = H[(size_t)i * m1 + i];
        y[i] = (d != 0.0) ? s / d : 0.0;
    }
}

__global__ void k_set_g(double *g, int n, double beta) {
    int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < n) g[i] = (i == 0) ? beta : 0.0;
}

static int nchunk_for(int64_t n) {
    int64_t c = (n + 4095) / 4096;
    if (c > 1024) c = 1024;
    if (c < 1) c = 1;
    return (int)c;
}

// dots out[0..nvec) = V[0..nvec)^T w  (mode as in k_finish)
static void dots(Mesh &m, const double *V, size_t ld, int nvec, const double *w, double *out,
                 int mode) {
    const int64_t n = m.np;
    const int nch = nchunk_for(n);
    const int chunk = (int)((n + nch - 1) / nch);
    dim3 grid(nch, nvec);
    k_dot_parts<<<grid, RED_THREADS, 0, m.stream>>>(V, ld, w, n, chunk, m.part.p);
    BEM_CHECK_LAUNCH();
    k_finish<<<nvec, RED_THREADS, 0, m.stream>>>(m.part.p, nch, out, mode);
    BEM_CHECK_LAUNCH();
}

static double read_scalar(Mesh &m, const double *d) {
    BEM_CUDA(cudaMemcpyAsync(m.h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, m.stream));
    BEM_CUDA(cudaStreamSynchronize(m.stream));
    return m.h_pinned[0];
}

double norm2(Mesh &m, const double *w) {
    dots(m, w, 0, 1, w, m.red.p, 2);
    return read_scalar(m, m.red.p);
}

// Solve A x = b (sorted order).  x holds the initial guess on entry.
int gmres_solve(Mesh &m, const double *b, double *x, bool transpose, bem_solve_stats *st) {
    const int64_t n = m.np;
    const int mr = std::max(1, m.opt.gmres_restart);
    const int m1 = mr + 1;
    const size_t ld = (size_t)n;
    cudaStream_t s = m.stream;
    if (m.V.n < (size_t)m1 * ld) m.V.alloc((size_t)m1 * ld);
    if (m.H.n < (size_t)m1 * mr) m.H.alloc((size_t)m1 * mr);
    if (m.gv.n < (size_t)m1) m.gv.alloc(m1);
    if (m.cs.n < (size_t)mr) { m.cs.alloc(mr); m.sn.alloc(mr); }
    if (m.yv.n < (size_t)mr) m.yv.alloc(mr);
    if (m.hv.n < (size_t)m1 + 2) m.hv.alloc(m1 + 2);
    const int nb = cdiv(n, 256);
    auto apply = [&](const double *in, double *out) {
        if (!transpose) matvec_sorted(m, in, out);
        else {
            matvec_t_sorted(m, in, out);
        }
    };
    const double bnorm = norm2(m, b);
    int it = 0, restarts = 0;
    double rec = 1.0;
    bool conv = false, stagnated = false;
    std::vector<double> hist;
    if (bnorm == 0.0) {
        BEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        rec = 0.0;
        conv = true;
    }
    bool x_zero = false;
    {
        // detect an all-zero initial guess to skip one product
        const double xn = conv ? 0.0 : norm2(m, x);
        x_zero = (xn == 0.0);
    }
    while (!conv && it < m.opt.max_iter && !stagnated) {
        double *V0 = m.V.p;
        if (x_zero) {
            BEM_CUDA(cudaMemcpyAsync(V0, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            apply(x, V0);
            k_axpby<<<nb, 256, 0, s>>>(1.0, b, -1.0, V0, V0, n);
            BEM_CHECK_LAUNCH();
        }
        const double beta = norm2(m, V0);
        rec = beta / bnorm;
        if (rec <= m.opt.tol) {
            conv = true;
            break;
        }
        // V0 /= beta, with beta read on the device (norm2 left it in red[0])
        k_scale_by_inv<<<nb, 256, 0, s>>>(V0, m.red.p, n);
        BEM_CHECK_LAUNCH();
        k_set_g<<<1, 64, 0, s>>>(m.gv.p, m1, beta);
        BEM_CHECK_LAUNCH();
        int k = 0;
        for (int j = 0; j < mr; ++j) {
            double *w = m.V.p + (size_t)(j + 1) * ld;
            apply(m.V.p + (size_t)j * ld, w);
            ++it;
            // CGS2: two passes of classical Gram-Schmidt
            dots(m, m.V.p, ld, j + 1, w, m.hv.p, 0);
            k_multi_axpy<<<nb, 256, 0, s>>>(m.V.p, ld, j + 1, m.hv.p, -1.0, w, n);
            BEM_CHECK_LAUNCH();
            dots(m, m.V.p, ld, j + 1, w, m.yv.p, 0);
            k_multi_axpy<<<nb, 256, 0, s>>>(m.V.p, ld, j + 1, m.yv.p, -1.0, w, n);
            BEM_CHECK_LAUNCH();
            k_axpby<<<1, 64, 0, s>>>(1.0, m.hv.p, 1.0, m.yv.p, m.hv.p, j + 1);
            BEM_CHECK_LAUNCH();
            dots(m, w, 0, 1, w, m.hv.p + j + 1, 2);
            k_givens<<<1, 1, 0, s>>>(m.H.p, m1, m.hv.p, j, m.cs.p, m.sn.p, m.gv.p, 1.0 / bnorm,
                                     m.red.p);
            BEM_CHECK_LAUNCH();
            k_scale_by<<<nb, 256, 0, s>>>(w, m.red.p + 1, n);
            BEM_CHECK_LAUNCH();
            rec = read_scalar(m, m.red.p);
            hist.push_back(rec);
            k = j + 1;
            if (!(rec == rec)) {  // NaN
                stagnated = true;
                break;
            }
            if (rec <= m.opt.tol || it >= m.opt.max_iter) break;
            const size_t hs = hist.size();
            if (hs > 60 && rec > 0.5 * hist[hs - 51]) {
                stagnated = true;
                break;
            }
        }
        k_backsolve<<<1, 1, 0, s>>>(m.H.p, m1, m.gv.p, k, m.yv.p);
        BEM_CHECK_LAUNCH();
        k_multi_axpy<<<nb, 256, 0, s>>>(m.V.p, ld, k, m.yv.p, 1.0, x, n);
        BEM_CHECK_LAUNCH();
        x_zero = false;
        if (rec <= m.opt.tol) conv = true;
        else ++restarts;
    }
    double true_res = rec;
    if (st) {
        // true residual from one more product
        apply(x, m.ys.p);
        k_axpby<<<nb, 256, 0, s>>>(1.0, b, -1.0, m.ys.p, m.ys.p, n);
        BEM_CHECK_LAUNCH();
        true_res = (bnorm > 0) ? norm2(m, m.ys.p) / bnorm : 0.0;
        st->iterations = it;
        st->restarts = restarts;
        st->converged = conv ? 1 : 0;
        st->resid = rec;
        st->true_resid = true_res;
    }
    BEM_CUDA(cudaStreamSynchronize(s));
    return conv ? BEM_OK : BEM_ENOCONV;
}

// dG = 4 pi 332.0637 / (2 eps_in) * (C^T q) . sigma
double energy_from_ctq(Mesh &m, const double *sig_s) {
    const int64_t n = m.np;
    const int nch = nchunk_for(n);
    const int chunk = (int)((n + nch - 1) / nch);
    dim3 grid(nch, 1);
    k_dot_parts<<<grid, RED_THREADS, 0, m.stream>>>(m.ctq.p, 0, sig_s, n, chunk, m.part.p);
    BEM_CHECK_LAUNCH();
    k_finish<<<1, RED_THREADS, 0, m.stream>>>(m.part.p, nch, m.red.p + 2, 0);
    BEM_CHECK_LAUNCH();
    const double ctqs = read_scalar(m, m.red.p + 2);
    return FOUR_PI * KCAL / (2.0 * m.eps_in) * ctqs;
}

// dG = 4 pi 332.0637 / (2 eps_in) * q . phi   (phi = C sigma, G = 1/(4 pi r))
double energy_from_phi(Mesh &m, const double *phi_s) {
    const int64_t n = m.nc;
    const int nch = nchunk_for(n);
    const int chunk = (int)((n + nch - 1) / nch);
    dim3 grid(nch, 1);
    k_dot_parts<<<grid, RED_THREADS, 0, m.stream>>>(m.q64.p, 0, phi_s, n, chunk, m.part.p);
    BEM_CHECK_LAUNCH();
    k_finish<<<1, RED_THREADS, 0, m.stream>>>(m.part.p, nch, m.red.p + 2, 0);
    BEM_CHECK_LAUNCH();
    const double qphi = read_scalar(m, m.red.p + 2);
    return FOUR_PI * KCAL / (2.0 * m.eps_in) * qphi;
}

void axpby(Mesh &m, double a, const double *x, double b, const double *y, double *out, int64_t n) {
    k_axpby<<<cdiv(n, 256), 256, 0, m.stream>>>(a, x, b, y, out, n);
    BEM_CHECK_LAUNCH();
}

}  // namespace bem
