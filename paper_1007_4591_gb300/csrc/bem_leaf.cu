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

template <class T>
void p2m_leaves(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src, const int *qpanel,
                const double *dens, int p, int cs, T inv_h, T *M, cudaStream_t s) {
    if (nleaf > 0) p2m_dispatch<T>(tv, nleaf, sk, src, qpanel, dens, p, cs, inv_h, M, s);
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
