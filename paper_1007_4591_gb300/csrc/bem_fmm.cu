// Fast multipole passes of the FMM-BEM matrix-vector product (Sec. 2.3):
// P2M, M2M (upward sweep), M2L, L2L (downward sweep), L2P + P2P (evaluation).
//
// Expansions use complex solid harmonics in the normalisation
//   R_n^m(r) = regular, I_n^m(r) = irregular,  1/|x-y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x),
// generated by the Cartesian recurrences
//   R_0^0 = 1,  R_m^m = -(x+iy)/(2m) R_{m-1}^{m-1},
//   R_n^m = ((2n-1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n+m)(n-m)),
//   I_0^0 = 1/r, I_m^m = -(2m-1)(x+iy)/r^2 I_{m-1}^{m-1},
//   I_n^m = ((2n-1) z I_{n-1}^m - (n-1-m)(n-1+m) I_{n-2}^m) / r^2,
// with X_n^{-m} = (-1)^m conj(X_n^m).  In these units the translations are
// plain convolutions:
//   P2M  M_n^m  = sum_i s_i conj(R_n^m(y_i - z))
//   M2M  M'_n^m = sum_{k,l} conj(R_k^l(z_c - z_p)) M_{n-k}^{m-l}
//   M2L  L_k^l  = (-1)^k sum_{n,m} M_n^m I_{n+k}^{m+l}(z_t - z_s)
//   L2L  L'_k^l = sum_{n,m} L_n^m conj(R_{n-k}^{m-l}(z_c - z_p))
//   L2P  phi(x) = sum L_n^m conj(R_n^m(x - z)),
//        grad phi = (-Re L'_1^1, -Im L'_1^1, Re L'_1^0),  L'_1^l = sum L_n^m conj(R_{n-1}^{m-l}(x - z)).
// Multipoles are stored divided by h^n and locals multiplied by h^(k+1)
// (h = cell size), which makes M2M, M2L and L2L independent of the level:
// the offsets are (+-1/4)^3 for parent/child and integer vectors in
// [-3,3]^3 for M2L.  The paper rotates every expansion before an axial
// translation (Sec. 4.3); here the 343 offset classes are tabulated once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

#include "bem_device.cuh"

namespace bem {

// ------------------------------------------------------------- constants
__constant__ double c_rinv_d[MAXP + 1][MAXP + 1];  // 1/((n+m)(n-m))
__constant__ float c_rinv_f[MAXP + 1][MAXP + 1];
__constant__ double c_inv2m_d[MAXP + 1];            // 1/(2m)
__constant__ float c_inv2m_f[MAXP + 1];
__constant__ double c_pow2n_d[2 * MAXP + 2];        // 2^-j
__constant__ float c_pow2n_f[2 * MAXP + 2];
__constant__ unsigned char c_tri_n[(MAXP + 1) * (MAXP + 2) / 2];
__constant__ unsigned char c_tri_m[(MAXP + 1) * (MAXP + 2) / 2];

template <class T> struct K;
template <> struct K<float> {
    __device__ static float rinv(int n, int m) { return c_rinv_f[n][m]; }
    __device__ static float inv2m(int m) { return c_inv2m_f[m]; }
    __device__ static float pow2n(int j) { return c_pow2n_f[j]; }
};
template <> struct K<double> {
    __device__ static double rinv(int n, int m) { return c_rinv_d[n][m]; }
    __device__ static double inv2m(int m) { return c_inv2m_d[m]; }
    __device__ static double pow2n(int j) { return c_pow2n_d[j]; }
};

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// r^-3 from r^2.  FP32: 2^(-1.5 log2 r^2) with the approximate base-2
// logarithm and exponential of the special-function unit (two of its
// operations and one multiply, against a reciprocal square root and two
// multiplies); both carry ~2^-22 error, about that of the cubed rsqrt.
__device__ __forceinline__ float lg2a(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rinv3(float r2) { return ex2a(-1.5f * lg2a(r2)); }
__device__ __forceinline__ double rinv3(double r2) {
    const double ri = rsqrt(r2);
    return ri * ri * ri;
}

// Regular solid harmonics R_n^m(x,y,z), 0 <= m <= n <= p, handed to emit(n, m, re, im).
template <class T, class F>
__device__ __forceinline__ void regular_solid(T x, T y, T z, int p, F &&emit) {
    const T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            const T f = -K<T>::inv2m(m);
            const T nre = f * (x * dre - y * dim), nim = f * (x * dim + y * dre);
            dre = nre;
            dim = nim;
        }
        emit(m, m, dre, dim);
        if (m + 1 > p) break;
        T are = dre, aim = dim;
        T bre = z * dre, bim = z * dim;
        emit(m + 1, m, bre, bim);
        for (int n = m + 2; n <= p; ++n) {
            const T c1 = (T)(2 * n - 1) * z, c2 = K<T>::rinv(n, m);
            const T nre = (c1 * bre - r2 * are) * c2, nim = (c1 * bim - r2 * aim) * c2;
            are = bre;
            aim = bim;
            bre = nre;
            bim = nim;
            emit(n, m, bre, bim);
        }
    }
}

__device__ __forceinline__ int cre(int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); }

// compact real layout -> full-m complex array X[n][m + p], stride W = 2p+1
template <class T>
__device__ __forceinline__ void load_full(const T *src, int p, cpx<T> *dst) {
    const int W = 2 * p + 1;
    const int tot = (p + 1) * W;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int n = idx / W, mm = idx - n * W - p;
        cpx<T> v;
        v.x = 0;
        v.y = 0;
        const int am = mm < 0 ? -mm : mm;
        if (am <= n) {
            T re = src[cre(n, am)], im = am == 0 ? (T)0 : src[n * n + 2 * am];
            if (mm < 0) {
                const T sg = (am & 1) ? (T)-1 : (T)1;
                re *= sg;
                im *= -sg;
            }
            v.x = re;
            v.y = im;
        }
        dst[idx] = v;
    }
}

// ------------------------------------------------------------------- P2M
// ------------------------------------------------------------------- M2M
// Parents [first, last) gather their children's multipoles.
template <class T>
__global__ void k_m2m(TreeView tv, int first, const cpx<T> *Rtab, int p, int cs, T *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1;
    cpx<T> *Mc = reinterpret_cast<cpx<T> *>(smraw);
    cpx<T> *Rd = Mc + (p + 1) * W;
    const int cell = first + blockIdx.x;
    const int nc = (p + 1) * (p + 1);
    const int ntri = (p + 1) * (p + 2) / 2;
    const int t = threadIdx.x;
    int n = 0, m = 0;
    if (t < ntri) {
        n = c_tri_n[t];
        m = c_tri_m[t];
    }
    cpx<T> acc;
    acc.x = 0;
    acc.y = 0;
    const int cb = tv.child_beg[cell], ce = tv.child_end[cell];
    for (int c = cb; c < ce; ++c) {
        __syncthreads();
        load_full<T>(M + (size_t)c * cs, p, Mc);
        const int4 q = tv.ijk[c];
        const int oct = (q.x & 1) | ((q.y & 1) << 1) | ((q.z & 1) << 2);
        const cpx<T> *R = Rtab + (size_t)oct * (p + 1) * W;
        for (int idx = t; idx < (p + 1) * W; idx += blockDim.x) Rd[idx] = R[idx];
        __syncthreads();
        if (t < ntri) {
            for (int k = 0; k <= n; ++k) {
                const T s = K<T>::pow2n(n - k);
                const int lmin = max(-k, m - (n - k)), lmax = min(k, m + (n - k));
                cpx<T> part;
                part.x = 0;
                part.y = 0;
                for (int l = lmin; l <= lmax; ++l)
                    cmac_conjb<T>(part, Mc[(n - k) * W + (m - l) + p], Rd[k * W + l + p]);
                acc.x += s * part.x;
                acc.y += s * part.y;
            }
        }
    }
    if (t < ntri) {
        T *out = M + (size_t)cell * cs;
        if (m == 0) out[n * n] = acc.x;
        else {
            out[n * n + 2 * m - 1] = acc.x;
            out[n * n + 2 * m] = acc.y;
        }
    }
}

// ------------------------------------------------------------------- M2L
// Cells [first, first + gridDim.x) receive their interaction lists; the local
// expansion is overwritten (L2L adds the parent's part afterwards).
template <class T>
__global__ void k_m2l(TreeView tv, int first, const cpx<T> *Itab, int p, int cs, const T *M, T *L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1, W2 = 4 * p + 1;
    cpx<T> *Ms = reinterpret_cast<cpx<T> *>(smraw);
    cpx<T> *It = Ms + (p + 1) * W;
    const int cell = first + blockIdx.x;
    const int nc = (p + 1) * (p + 1);
    const int ntri = (p + 1) * (p + 2) / 2;
    const int t = threadIdx.x;
    int k = 0, l = 0;
    if (t < ntri) {
        k = c_tri_n[t];
        l = c_tri_m[t];
    }
    cpx<T> acc;
    acc.x = 0;
    acc.y = 0;
    const int eb = tv.m2l_off[cell], ee = tv.m2l_off[cell + 1];
    const int itot = (2 * p + 1) * W2;
    for (int e = eb; e < ee; ++e) {
        __syncthreads();
        load_full<T>(M + (size_t)tv.m2l_src[e] * cs, p, Ms);
        const cpx<T> *I = Itab + (size_t)tv.m2l_ofs[e] * itot;
        for (int idx = t; idx < itot; idx += blockDim.x) It[idx] = I[idx];
        __syncthreads();
        if (t < ntri) {
            for (int n = 0; n <= p; ++n) {
                const cpx<T> *Irow = It + (n + k) * W2 + l + 2 * p;
                const cpx<T> *Mrow = Ms + n * W + p;
                for (int m = -n; m <= n; ++m) cmac<T>(acc, Mrow[m], Irow[m]);
            }
        }
    }
    if (t < ntri) {
        const T sg = (k & 1) ? (T)-1 : (T)1;
        T *out = L + (size_t)cell * cs;
        if (l == 0) out[k * k] = sg * acc.x;
        else {
            out[k * k + 2 * l - 1] = sg * acc.x;
            out[k * k + 2 * l] = sg * acc.y;
        }
    }
}

// ------------------------------------------------------------------- L2L
// Children [first, first + gridDim.x) add their parent's local expansion.
template <class T>
__global__ void k_l2l(TreeView tv, int first, const cpx<T> *Rtab, int p, int cs, T *L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1;
    cpx<T> *Lp = reinterpret_cast<cpx<T> *>(smraw);
    cpx<T> *Rd = Lp + (p + 1) * W;
    const int cell = first + blockIdx.x;
    const int nc = (p + 1) * (p + 1);
    const int ntri = (p + 1) * (p + 2) / 2;
    const int t = threadIdx.x;
    const int P = tv.parent[cell];
    load_full<T>(L + (size_t)P * cs, p, Lp);
    const int4 q = tv.ijk[cell];
    const int oct = (q.x & 1) | ((q.y & 1) << 1) | ((q.z & 1) << 2);
    const cpx<T> *R = Rtab + (size_t)oct * (p + 1) * W;
    for (int idx = t; idx < (p + 1) * W; idx += blockDim.x) Rd[idx] = R[idx];
    __syncthreads();
    if (t < ntri) {
        const int k = c_tri_n[t], l = c_tri_m[t];
        cpx<T> acc;
        acc.x = 0;
        acc.y = 0;
        for (int n = k; n <= p; ++n) {
            const int j = n - k;
            const int mmin = max(-n, l - j), mmax = min(n, l + j);
            for (int mm = mmin; mm <= mmax; ++mm)
                cmac_conjb<T>(acc, Lp[n * W + mm + p], Rd[j * W + (mm - l) + p]);
        }
        const T s = K<T>::pow2n(k + 1);
        T *out = L + (size_t)cell * cs;
        if (l == 0) out[k * k] += s * acc.x;
        else {
            out[k * k + 2 * l - 1] += s * acc.x;
            out[k * k + 2 * l] += s * acc.y;
        }
    }
}

// ------------------------------------------------------------------- L2P
// L2P: one CTA per leaf, sized to the leaves' average number of targets
// (l2p_threads); the local expansion is expanded into the full
// (n, m = -n..n) array in shared memory.
template <class T, int TGT>
__global__ void __launch_bounds__(128) k_l2p(TreeView tv, const typename V4T<T>::t *tgt, const typename V4T<T>::t *nrm,
                      int p, int cs, T inv_h, const T *L, T *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1;
    cpx<T> *Lf = reinterpret_cast<cpx<T> *>(smraw);
    const int leaf = blockIdx.x;
    constexpr bool DN = TGT == TGT_CEN_DN || TGT == TGT_QUAD_DN;  // normal field, else potential
    const int *beg = TGT == TGT_CEN_DN ? tv.cen_beg : (TGT == TGT_CHG_PHI ? tv.chg_beg : tv.qp_beg);
    const int b = beg[leaf], e = beg[leaf + 1];
    if (b == e) return;
    load_full<T>(L + (size_t)(tv.leaf0 + leaf) * cs, p, Lf);
    __syncthreads();
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const typename V4T<T>::t r = tgt[i];
        const T x = r.x * inv_h, y = r.y * inv_h, z = r.z * inv_h;
        if (DN) {
            cpx<T> a10, a11;
            a10.x = a10.y = a11.x = a11.y = 0;
            regular_solid<T>(x, y, z, p - 1, [&](int n, int m, T re, T im) {
                const cpx<T> *row = Lf + (n + 1) * W + p;
                cpx<T> R;
                R.x = re;
                R.y = im;
                cmac_conjb<T>(a10, row[m], R);
                cmac_conjb<T>(a11, row[m + 1], R);
                if (m > 0) {
                    const T sg = (m & 1) ? (T)-1 : (T)1;
                    cpx<T> Rn;  // conj(R_n^{-m}) = (-1)^m R_n^m
                    Rn.x = sg * re;
                    Rn.y = sg * im;
                    cmac<T>(a10, row[-m], Rn);
                    cmac<T>(a11, row[1 - m], Rn);
                }
            });
            const typename V4T<T>::t nn = nrm[i];
            const T s2 = inv_h * inv_h;
            out[i] = s2 * (-nn.x * a11.x - nn.y * a11.y + nn.z * a10.x);
        } else {
            cpx<T> a00;
            a00.x = a00.y = 0;
            regular_solid<T>(x, y, z, p, [&](int n, int m, T re, T im) {
                const cpx<T> *row = Lf + n * W + p;
                cpx<T> R;
                R.x = re;
                R.y = im;
                cmac_conjb<T>(a00, row[m], R);
                if (m > 0) {
                    const T sg = (m & 1) ? (T)-1 : (T)1;
                    cpx<T> Rn;
                    Rn.x = sg * re;
                    Rn.y = sg * im;
                    cmac<T>(a00, row[-m], Rn);
                }
            });
            out[i] = inv_h * a00.x;
        }
    }
}

// ------------------------------------------------------------------- P2P
// Near field of one target leaf: all source points of the adjacent leaves
// (and the leaf itself), staged through shared memory with coordinates moved
// into the target leaf's frame.  G threads share one target and split each
// tile; a pair with coincident points (the collocation point against its own
// panel's centroid node) contributes exactly zero: d = 0 gives n.d = 0 and
// r^2 = eps, so the product stays finite.
constexpr int P2P_THREADS = 256;

template <class T> struct P2PEps;
template <> struct P2PEps<float> { static constexpr float v = 1e-20f; };
template <> struct P2PEps<double> { static constexpr double v = 1e-40; };

// Geometric factors of one (collocation point, source point) pair of the K'
// near field: n.d and |d|^-3 with d = c - y.  The near-singular table
// replays exactly this arithmetic, so keep every use on this one function.
template <class T>
__device__ __forceinline__ void dn_pair(T dx, T dy, T dz, T nx, T ny, T nz, T &nd, T &ri3) {
    const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, P2PEps<T>::v)));
    nd = fma(nx, dx, fma(ny, dy, nz * dz));
    ri3 = rinv3(r2);
}

// Strength records of a pass's near field, in pairs of sources: the sources
// of leaf S occupy pairs [P_S, P_S + ceil(n_S / 2)), P_S = ceil((beg_S + S) / 2)
// (every leaf starts on a whole pair, and P_S + ceil(n_S / 2) <= P_{S+1}),
// pair p as out[2p] = (x0, x1, y0, y1), out[2p + 1] = (z0, z1, s0, s1) with the
// leaf-relative coordinates and the strengths s = A_j w_q dens[panel] for
// quadrature points or s = q_k (or dens[k]) for charges; an odd leaf's last
// pair has a zero partner.  One CTA (an even number of threads) per leaf.
template <class T, int SRC>
__global__ void k_strength_pairs(TreeView tv, const typename V4T<T>::t *rec, const int *qpanel, const double *dens,
                                 typename V4T<T>::t *out) {
    using V4 = typename V4T<T>::t;
    const int S = blockIdx.x;
    const int *sb_ = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int b = sb_[S], n = sb_[S + 1] - b;
    const int64_t P = ((int64_t)b + S + 1) >> 1;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        T x = 0, y = 0, z = 0, w = 0;
        if (i < n) {
            const V4 r = rec[b + i];
            x = r.x;
            y = r.y;
            z = r.z;
            w = src_strength<T, SRC>(r.w, (int64_t)b + i, qpanel, dens);
        }
        // the odd lane's values go to its even neighbour (zero past the end)
        const T px = __shfl_down_sync(0xffffffffu, x, 1), py = __shfl_down_sync(0xffffffffu, y, 1);
        const T pz = __shfl_down_sync(0xffffffffu, z, 1), pw = __shfl_down_sync(0xffffffffu, w, 1);
        if (!(threadIdx.x & 1) && i < n) {
            V4 a, c;
            a.x = x;
            a.y = px;
            a.z = y;
            a.w = py;
            c.x = z;
            c.y = pz;
            c.z = w;
            c.w = pw;
            const int64_t pr = P + (i >> 1);
            out[2 * pr] = a;
            out[2 * pr + 1] = c;
        }
    }
}

// y = x + Ehat (far + near64) / (4 pi), near64 already holding the table's
// correction: the collocation product's epilogue where L2P cannot carry it.
template <class T>
__global__ void k_apply_far_near(const double *x, const T *far, const double *near64, double ehat, int64_t n,
                                 double *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = near64 ? near64[i] : 0.0;
    if (far) v += (double)far[i];
    y[i] = x[i] + ehat * (v * (1.0 / FOUR_PI));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16-byte copy global -> shared (ok = false writes zero, src-size 0)
__device__ __forceinline__ void cp_async_16(void *dst, const void *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

// Two lanes of T: packed FP32 instructions on sm_100+ (per component the
// same rounding as the scalar fmaf / fadd / fmul), plain pairs for FP64.
template <class T> struct Pk;
template <> struct Pk<float> {
    using v = float2;
    __device__ static v mk(float a, float b) { return make_float2(a, b); }
    __device__ static v add(v a, v b) { return __fadd2_rn(a, b); }
    __device__ static v mul(v a, v b) { return __fmul2_rn(a, b); }
    __device__ static v fma(v a, v b, v c) { return __ffma2_rn(a, b, c); }
    // r^-3 per lane, the arithmetic of rinv3 (the multiply packed)
    __device__ static v rinv3(v r2) {
        const v e = __fmul2_rn(make_float2(lg2a(r2.x), lg2a(r2.y)), make_float2(-1.5f, -1.5f));
        return make_float2(ex2a(e.x), ex2a(e.y));
    }
};
template <> struct Pk<double> {
    using v = double2;
    __device__ static v mk(double a, double b) { return make_double2(a, b); }
    __device__ static v add(v a, v b) { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ static v mul(v a, v b) { return make_double2(a.x * b.x, a.y * b.y); }
    __device__ static v fma(v a, v b, v c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
    __device__ static v rinv3(v r2) { return make_double2(::bem::rinv3(r2.x), ::bem::rinv3(r2.y)); }
};

// Near field of one target leaf: every source point of the adjacent leaves
// (and the leaf itself), streamed through shared memory in tiles of source
// pairs, coordinates moved into the target leaf's frame.  The source pairs
// come from the pair records of k_strength_pairs, (x0,x1,y0,y1) and
// (z0,z1,s0,s1), so one packed instruction evaluates a target against two
// sources; a neighbour leaf's pairs are a contiguous run (its odd partner has
// weight zero).
// Staging: each thread owns PPT pair slots of every tile.  After the tile's
// barrier it copies the records of its slots of the next tile with cp.async
// into the second of two buffers, computes the current tile, then rewrites its
// own slots in place into the target leaf's frame, -(y + o) (the loop then
// forms c - (y + o) as c + (-(y + o)), the same value, with plain packed
// adds).  A thread finds the neighbour leaf of each of its pairs by a forward
// walk over the leaves' running pair counts (its pairs increase monotonically).
// Thread mapping of the arithmetic: targets are taken P2P_TPT at a time into
// groups; the threads split into ngroups x G (G = threads / ngroups, any
// integer), each thread owning P2P_TPT targets and a 1/G share of the source
// pairs of each tile (a tile holds a whole number of pairs per thread).  Tile
// sums go into a second accumulator; the G partial sums of a target are added
// in a fixed order at the end.  A pair of coincident points (a collocation
// point and its own panel's centroid node) gives d = 0, n.d = 0 and
// r^2 = eps, a finite zero; so does a zero partner placed at a target.
// Targets per thread: 3 in FP32 (measured against 4: the product 0.2883 vs
// 0.2947 ms, no register spills at 64 registers, and leaves of ~17 targets
// pad to 18 instead of 20), 2 in FP64.
template <class T> struct P2PTpt;
template <> struct P2PTpt<float> { static constexpr int v = 3; };
template <> struct P2PTpt<double> { static constexpr int v = 2; };
// Pair slots per thread and tile: FP32 tiles of 384 pairs for 128 threads
// (24 KB for the two buffers: 8 CTAs per SM) and 512 for 256 threads.
template <class T, int NT> struct P2PPpt { static constexpr int v = 1; };
template <> struct P2PPpt<float, 128> { static constexpr int v = 3; };
template <> struct P2PPpt<float, 256> { static constexpr int v = 2; };

// Dynamic shared memory of k_p2p: two buffers of pair records.
template <class T, int NT>
constexpr size_t p2p_smem() {
    return (size_t)2 * 2 * NT * P2PPpt<T, NT>::v * sizeof(typename V4T<T>::t);
}

// A neighbour leaf of the target leaf: its offset in the target leaf's frame
// and the index of its first source pair less its start in the leaf's
// concatenated pair list.
template <class T>
struct alignas(4 * sizeof(T)) NbSeg {
    T ox, oy, oz;
    int base;
};

// Work list of the near-field kernel (k_p2p_list): per CTA, in launch order,
// hdr[3b] = (neighbour leaves nn, source pairs, first record, 0),
// hdr[3b + 1] = (first and end centroid, first and end quadrature point),
// hdr[3b + 2] = (first and end charge, 0, 0), and the records
// rec[first + k] = (P_S - pc_k, pc_k << 9 | cell offset of neighbour k) with
// P_S the first pair of leaf S (k_strength_pairs), pc_k the pairs of
// neighbours 0..k-1 and the offset's components + 2 in 3-bit fields.  Lists
// of one-cell separation keep 27 record slots per CTA (first = 27 b, so a CTA
// loads header and records in one round), wider ones are packed.
struct P2PList {
    const int4 *hdr;
    const int2 *rec;
};

// One CTA (128 threads) per launch slot b: the records of leaf p2p_order[b];
// first[b] is the slot's first record.
template <int SRC>
__global__ void k_p2p_list(TreeView tv, const int64_t *first, int4 *hdr, int2 *rec) {
    __shared__ int s_pc[129];
    const int b = blockIdx.x, leaf = tv.p2p_order[b];
    const int nb0 = tv.nbr_off[leaf], nn = tv.nbr_off[leaf + 1] - nb0;
    const int *sb_ = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int k = threadIdx.x;
    int S = 0;
    if (k < nn) {
        S = tv.nbr[nb0 + k];
        s_pc[k + 1] = (sb_[S + 1] - sb_[S] + 1) >> 1;
    }
    __syncthreads();
    if (k == 0) {
        s_pc[0] = 0;
        for (int j = 0; j < nn; ++j) s_pc[j + 1] += s_pc[j];
    }
    __syncthreads();
    const int64_t f = first[b];
    if (k < nn) {
        const int4 ct = tv.ijk[tv.leaf0 + leaf], cs = tv.ijk[tv.leaf0 + S];
        const int d = (cs.x - ct.x + 2) | ((cs.y - ct.y + 2) << 3) | ((cs.z - ct.z + 2) << 6);
        rec[f + k] = make_int2((int)(((int64_t)sb_[S] + S + 1) >> 1) - s_pc[k], (s_pc[k] << 9) | d);
    }
    if (k == 0) {
        hdr[3 * b] = make_int4(nn, s_pc[nn], (int)f, 0);
        hdr[3 * b + 1] = make_int4(tv.cen_beg[leaf], tv.cen_beg[leaf + 1], tv.qp_beg[leaf], tv.qp_beg[leaf + 1]);
        hdr[3 * b + 2] = make_int4(tv.chg_beg[leaf], tv.chg_beg[leaf + 1], 0, 0);
    }
}

// With tab.out64 set (the collocation K' product) each target's value goes
// out in FP64 together with 4 pi times its row of the near-singular table
// applied to tab.x: out64_i = near_i + 4 pi sum_e val_e x[col_e].
struct NearTab {
    const int *off, *col;
    const double *val, *x;
    double *out64;
};

// NB: the most neighbour leaves a leaf has (27 for one-cell separation, 125
// for the charge tree's two cells).
template <class T, int SRC, int TGT, int NT, int NB = 27>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 1024 / NT : 1)
k_p2p(P2PList wl, const typename V4T<T>::t *tgt, const typename V4T<T>::t *nrm,
      const typename V4T<T>::t *src, T h, T *out, NearTab tab) {
    using V4 = typename V4T<T>::t;
    using P = Pk<T>;
    using v2 = typename P::v;
    static_assert(NB <= NT, "one thread per neighbour leaf in the set-up");
    constexpr int P2P_TPT = P2PTpt<T>::v;
    constexpr int PPT = P2PPpt<T, NT>::v;
    constexpr int TP = NT * PPT;                 // pair slots per buffer
    constexpr int NCP = (int)(sizeof(V4) / 16);  // 16-byte copies per record
    constexpr int MAXT = (NT / 4) * P2P_TPT;     // targets per pass (G >= 4)
    extern __shared__ __align__(32) unsigned char p2p_sm[];
    V4 *shA = reinterpret_cast<V4 *>(p2p_sm);  // [2][TP] (x0,x1,y0,y1)
    V4 *shB = shA + 2 * TP;                    // [2][TP] (z0,z1,s0,s1)
    __shared__ T s_part[NT * P2P_TPT];
    __shared__ int s_pc[NB + 1];
    __shared__ NbSeg<T> s_seg[NB];
    __shared__ int s_row[MAXT + 1];  // the pass's table row offsets
    constexpr bool DN = TGT == TGT_CEN_DN || TGT == TGT_QUAD_DN;  // normal field, else potential
    // the CTA's header and neighbour records: one round of independent loads
    const int4 h0 = wl.hdr[3 * blockIdx.x];
    const int4 h1 = wl.hdr[3 * blockIdx.x + 1 + (TGT != TGT_CEN_DN && TGT != TGT_QUAD_DN)];
    int2 r = make_int2(0, 0);
    if (NB == 27 && threadIdx.x < NB) r = wl.rec[27 * (int64_t)blockIdx.x + threadIdx.x];
    const int nn = h0.x;
    const int tb = TGT == TGT_QUAD_DN ? h1.z : h1.x, te = TGT == TGT_QUAD_DN ? h1.w : h1.y;
    if (tb == te) return;
    if (NB != 27 && threadIdx.x < nn) r = wl.rec[h0.z + threadIdx.x];
    if (threadIdx.x < nn) {
        s_pc[threadIdx.x] = r.y >> 9;
        // offsets of at most two cells: d h with |d| <= 2 is exact in T
        NbSeg<T> sg;
        sg.ox = (T)((r.y & 7) - 2) * h;
        sg.oy = (T)(((r.y >> 3) & 7) - 2) * h;
        sg.oz = (T)(((r.y >> 6) & 7) - 2) * h;
        sg.base = r.x;
        s_seg[threadIdx.x] = sg;
    }
    if (threadIdx.x == 0) s_pc[nn] = h0.y;
    __syncthreads();
    const int total = s_pc[nn];  // source pairs
    int kslot[PPT];              // neighbour leaf of each of this thread's slots
    // copies of this thread's slots of the tpr pairs from pair pb into buffer bf
    auto issue = [&](int pb, int tpr, int bf, int &k) {
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int u = threadIdx.x + NT * i;
            const int j = pb + u;
            if (u < tpr && j < total) {
                while (s_pc[k + 1] <= j) ++k;
                kslot[i] = k;
                const char *g = reinterpret_cast<const char *>(src + 2 * (int64_t)(s_seg[k].base + j));
                char *da = reinterpret_cast<char *>(shA + bf * TP + u);
                char *db = reinterpret_cast<char *>(shB + bf * TP + u);
#pragma unroll
                for (int c = 0; c < NCP; ++c) {
                    cp_async_16(da + 16 * c, g + 16 * c, true);
                    cp_async_16(db + 16 * c, g + sizeof(V4) + 16 * c, true);
                }
            }
        }
        cp_async_commit();
    };
    // this thread's slots, in place: -(y + o) for both sources of a pair
    auto convert = [&](int pb, int tpr, int bf) {
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int u = threadIdx.x + NT * i;
            const int j = pb + u;
            if (u < tpr && j < total) {
                const NbSeg<T> sg = s_seg[kslot[i]];
                V4 a = shA[bf * TP + u], b = shB[bf * TP + u];
                a.x = -(a.x + sg.ox);
                a.y = -(a.y + sg.ox);
                a.z = -(a.z + sg.oy);
                a.w = -(a.w + sg.oy);
                b.x = -(b.x + sg.oz);
                b.y = -(b.y + sg.oz);
                shA[bf * TP + u] = a;
                shB[bf * TP + u] = b;
            }
        }
    };
    const int ntgt = te - tb;
    const v2 EPS2 = P::mk(P2PEps<T>::v, P2PEps<T>::v);
    for (int t0 = 0; t0 < ntgt; t0 += MAXT) {
        if (t0 > 0) __syncthreads();  // the previous pass's buffers and partial sums are read
        const int nt = min(ntgt - t0, MAXT);
        const int ngroups = (nt + P2P_TPT - 1) / P2P_TPT;
        const int G = NT / ngroups;
        const int grp = threadIdx.x / G, g = threadIdx.x - grp * G;
        const bool active = grp < ngroups;
        // tiles of a whole number of pairs per thread of a group: every
        // thread makes the same number of steps between two barriers
        const int tpr = (TP / G) * G;
        const int ntile = (total + tpr - 1) / tpr;
        int kw = 0;
        if (tab.off) {  // the pass's table row offsets, copied ahead: nt + 1 of them
            for (int j = threadIdx.x; j <= nt; j += NT) {
                const unsigned d = (unsigned)__cvta_generic_to_shared(s_row + j);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(tab.off + tb + t0 + j)
                             : "memory");
            }
        }
        if (ntile > 0) issue(0, tpr, 0, kw);
        else cp_async_commit();
        v2 cx[P2P_TPT], cy[P2P_TPT], cz[P2P_TPT], nx[P2P_TPT], ny[P2P_TPT], nz[P2P_TPT];
        T outer[P2P_TPT];
#pragma unroll
        for (int q = 0; q < P2P_TPT; ++q) {
            const int ti = grp * P2P_TPT + q;
            T a = 0, b = 0, c = 0, d = 0, e = 0, f = 0;
            if (active && ti < nt) {
                const V4 cv = tgt[tb + t0 + ti];
                a = cv.x;
                b = cv.y;
                c = cv.z;
                if (DN) {
                    const V4 nv = nrm[tb + t0 + ti];
                    d = nv.x;
                    e = nv.y;
                    f = nv.z;
                }
            }
            cx[q] = P::mk(a, a);
            cy[q] = P::mk(b, b);
            cz[q] = P::mk(c, c);
            nx[q] = P::mk(d, d);
            ny[q] = P::mk(e, e);
            nz[q] = P::mk(f, f);
            outer[q] = 0;
        }
        cp_async_wait<0>();
        if (ntile > 0) convert(0, tpr, 0);
        for (int it = 0; it < ntile; ++it) {
            const int pb = it * tpr;
            const int bf = it & 1;
            const bool more = it + 1 < ntile;
            // tile it is in place everywhere, and every thread is done with
            // tile it - 1, whose buffer the next copies overwrite
            __syncthreads();
            if (more) issue(pb + tpr, tpr, bf ^ 1, kw);
            const V4 *cA = shA + bf * TP, *cB = shB + bf * TP;
            const int npair = min(tpr, total - pb);
            if (active) {
                v2 acc[P2P_TPT];
#pragma unroll
                for (int q = 0; q < P2P_TPT; ++q) acc[q] = P::mk(0, 0);
#pragma unroll 2
                for (int j = g; j < npair; j += G) {
                    const V4 a = cA[j], b = cB[j];  // -(y + o) and the strengths
                    const v2 yx = P::mk(a.x, a.y), yy = P::mk(a.z, a.w);
                    const v2 yz = P::mk(b.x, b.y), yw = P::mk(b.z, b.w);
#pragma unroll
                    for (int q = 0; q < P2P_TPT; ++q) {
                        const v2 dx = P::add(cx[q], yx), dy = P::add(cy[q], yy), dz = P::add(cz[q], yz);
                        const v2 r2 = P::fma(dx, dx, P::fma(dy, dy, P::fma(dz, dz, EPS2)));
                        if (DN) {
                            const v2 nd = P::fma(nx[q], dx, P::fma(ny[q], dy, P::mul(nz[q], dz)));
                            acc[q] = P::fma(P::mul(yw, nd), P::rinv3(r2), acc[q]);
                        } else {
                            acc[q] = P::fma(yw, P::mk(rsq(r2.x), rsq(r2.y)), acc[q]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < P2P_TPT; ++q) outer[q] += acc[q].x + acc[q].y;
            }
            if (more) {
                cp_async_wait<0>();
                convert(pb + tpr, tpr, bf ^ 1);
            }
        }
        __syncthreads();
        // the near-singular table rows of the pass's targets (collocation
        // product): all threads gather the rows' entries and the inputs they
        // take into the freed pair buffers, then each target runs its row
        constexpr int ECAP = (int)(p2p_smem<T, NT>() / (2 * sizeof(double)));
        double *ev = reinterpret_cast<double *>(p2p_sm), *ex = ev + ECAP;
        const int e0 = tab.off ? s_row[0] : 0, ne = tab.off ? s_row[nt] - e0 : 0;
        if (ne <= ECAP)
            for (int e = threadIdx.x; e < ne; e += NT) {
                ev[e] = tab.val[e0 + e];
                ex[e] = tab.x[tab.col[e0 + e]];
            }
#pragma unroll
        for (int q = 0; q < P2P_TPT; ++q) s_part[threadIdx.x * P2P_TPT + q] = outer[q];
        __syncthreads();
        if (threadIdx.x < nt) {
            const int gr = threadIdx.x / P2P_TPT, q = threadIdx.x - gr * P2P_TPT;
            T a = 0;
            for (int k = 0; k < G; ++k) a += s_part[(gr * G + k) * P2P_TPT + q];
            const int i = tb + t0 + threadIdx.x;
            if (tab.out64) {
                double c = 0.0;
                if (tab.off) {
                    const int ea = s_row[threadIdx.x], eb = s_row[threadIdx.x + 1];
                    if (ne <= ECAP)
                        for (int e = ea - e0; e < eb - e0; ++e) c = fma(ev[e], ex[e], c);
                    else
                        for (int e = ea; e < eb; ++e) c = fma(tab.val[e], tab.x[tab.col[e]], c);
                }
                tab.out64[i] = (double)(DN ? -a : a) + FOUR_PI * c;
            } else {
                out[i] = DN ? -a : a;
            }
        }
    }
}

// ------------------------------------------------------ transposed K' pass
// Dipole sources p_i = lam_i n_i at the collocation points.  The multipole
// of a dipole is its own degree-1 expansion D_1^0 = p_z,
// D_1^{+-1} = -+ (p_x -+ i p_y)/2 translated like an M2M:
//   M_n^m = sum_{l=-1..1} conj(R_{n-1}^{m-l}(c - z)) D_1^l,
// accumulated here while the recurrence emits R_k^l (scaled by 1/h).
template <class T>
__global__ void k_p2m_dipole(TreeView tv, const int *dbeg, const typename V4T<T>::t *rec,
                             const typename V4T<T>::t *nrm, const double *lam, int p, int cs,
                             T inv_h, T *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sh = reinterpret_cast<T *>(smraw);
    const int leaf = blockIdx.x;
    const int b = dbeg[leaf], e = dbeg[leaf + 1];
    const int nc = (p + 1) * (p + 1);
    constexpr int MAXACC = 10;
    T acc[MAXACC];
#pragma unroll
    for (int k = 0; k < MAXACC; ++k) acc[k] = 0;
    for (int base = b; base < e; base += blockDim.x) {
        const int i = base + threadIdx.x;
        T *row = sh + threadIdx.x * nc;
        for (int c = 0; c < nc; ++c) row[c] = 0;
        if (i < e) {
            const typename V4T<T>::t r = rec[i], nv = nrm[i];
            const T l = (T)lam[i] * inv_h;
            const T px = l * nv.x, py = l * nv.y, pz = l * nv.z;
            // D_1^0 = pz, D_1^1 = -(px - i py)/2, D_1^-1 = (px + i py)/2
            const T d1r = -px / 2, d1i = py / 2, dmr = px / 2, dmi = py / 2;
            regular_solid<T>(r.x * inv_h, r.y * inv_h, r.z * inv_h, p - 1, [&](int k, int l, T re, T im) {
                const int n = k + 1;
                // conj(R) = (re, -im); add conj(R) * D to M_n^m
                auto add = [&](int m, T dr, T di) {  // m >= 0
                    const T vr = re * dr + im * di, vi = re * di - im * dr;
                    if (m == 0) row[n * n] += vr;
                    else {
                        row[n * n + 2 * m - 1] += vr;
                        row[n * n + 2 * m] += vi;
                    }
                };
                add(l, pz, 0);
                add(l + 1, d1r, d1i);
                if (l >= 1) add(l - 1, dmr, dmi);
                if (l == 1) {
                    // R_k^{-1} = -conj(R_k^1): conj(R_k^{-1}) D_1^1 = -(re + i im)(d1r + i d1i)
                    row[n * n] += -(re * d1r - im * d1i);
                }
            });
        }
        __syncthreads();
        const int cnt = min((int)blockDim.x, e - base);
        int k = 0;
        for (int c = threadIdx.x; c < nc; c += blockDim.x, ++k) {
            T a = 0;
            for (int j = 0; j < cnt; ++j) a += sh[j * nc + c];
#pragma unroll
            for (int q = 0; q < MAXACC; ++q)
                if (q == k) acc[q] += a;
        }
        __syncthreads();
    }
    T *out = M + (size_t)(tv.leaf0 + leaf) * cs;
    int k = 0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x, ++k) {
#pragma unroll
        for (int q = 0; q < MAXACC; ++q)
            if (q == k) out[c] = acc[q];
    }
}

// Near field of the transposed product, organised like the forward kernel:
// one CTA per leaf T of collocation points; the quadrature points of the
// adjacent leaves are moved into T's frame exactly as the forward kernel
// moves them, so every pair value n.d |d|^-3 is bit-identical to the
// forward one (the transposed near-singular table then replaces it exactly).
// Each thread owns quadrature points and loops over T's collocation points
// (staged with their lam_i and normals); results go out with one atomic add
// per point and CTA.
template <class T>
__global__ void __launch_bounds__(P2P_THREADS)
k_p2p_t(TreeView tv, const int *dbeg, const typename V4T<T>::t *cen, const typename V4T<T>::t *nrm,
        const double *lam, const typename V4T<T>::t *qrec, T h, T *outq) {
    using V4 = typename V4T<T>::t;
    __shared__ V4 sc[P2P_THREADS], sn[P2P_THREADS];
    __shared__ int s_beg[28], s_cum[28];
    __shared__ T s_off[27][3];
    const int leaf = tv.p2p_order[blockIdx.x];
    const int tb = dbeg[leaf], te = dbeg[leaf + 1];
    if (tb == te) return;
    const int nb0 = tv.nbr_off[leaf], nn = tv.nbr_off[leaf + 1] - nb0;
    const int4 ct = tv.ijk[tv.leaf0 + leaf];
    if (threadIdx.x < nn) {
        const int S = tv.nbr[nb0 + threadIdx.x];
        const int4 cs = tv.ijk[tv.leaf0 + S];
        s_beg[threadIdx.x] = tv.qp_beg[S];
        s_cum[threadIdx.x + 1] = tv.qp_beg[S + 1] - tv.qp_beg[S];
        s_off[threadIdx.x][0] = (T)((double)(cs.x - ct.x) * (double)h);
        s_off[threadIdx.x][1] = (T)((double)(cs.y - ct.y) * (double)h);
        s_off[threadIdx.x][2] = (T)((double)(cs.z - ct.z) * (double)h);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_cum[0] = 0;
        for (int k = 0; k < nn; ++k) s_cum[k + 1] += s_cum[k];
    }
    __syncthreads();
    const int total = s_cum[nn];
    const int ntgt = te - tb;
    for (int t0 = 0; t0 < ntgt; t0 += P2P_THREADS) {
        const int nt = min(ntgt - t0, P2P_THREADS);
        __syncthreads();
        if (threadIdx.x < nt) {
            V4 c = cen[tb + t0 + threadIdx.x];
            c.w = (T)lam[tb + t0 + threadIdx.x];
            sc[threadIdx.x] = c;
            sn[threadIdx.x] = nrm[tb + t0 + threadIdx.x];
        }
        __syncthreads();
        for (int v = threadIdx.x; v < total; v += P2P_THREADS) {
            int lo = 0, hi = nn;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_cum[mid] <= v) lo = mid;
                else hi = mid;
            }
            const int qi = s_beg[lo] + (v - s_cum[lo]);
            V4 y = qrec[qi];
            y.x += s_off[lo][0];
            y.y += s_off[lo][1];
            y.z += s_off[lo][2];
            T acc = 0;
            for (int i = 0; i < nt; ++i) {
                const V4 c = sc[i], nv = sn[i];
                T nd, ri3;
                dn_pair<T>(c.x - y.x, c.y - y.y, c.z - y.z, nv.x, nv.y, nv.z, nd, ri3);
                acc = fma(c.w * nd, ri3, acc);
            }
            atomicAdd(outq + qi, -acc);
        }
    }
}

// z_j = 1/(4 pi) sum_q A_j w_q (far_q + near_q) over the points of panel j
template <class T>
__global__ void k_panel_reduce(const T *far, const T *near, const int *qp_of_panel,
                               const double *qw, int nq, int64_t np, double *out,
                               const double *area = nullptr) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double a = 0.0;
    for (int q = 0; q < nq; ++q) {
        const int k = qp_of_panel[j * nq + q];
        double v = near ? (double)near[k] : 0.0;
        if (far) v += (double)far[k];
        a += qw[k] * v;
    }
    // with area: the rule's average over the panel (weights qw / A_j)
    out[j] = (area ? a / area[j] : a) / FOUR_PI;
}

// ------------------------------------------------------ near-singular table
// For each collocation point i, the panels j close to it (centroid distance
// below 2.5 sqrt(A_i), which covers the panels sharing a vertex or an edge,
// plus i itself) get an FP64 correction
//   D_ij = 1/(4 pi) sum_q [ -A_j w_q (c_i - y_jq).n_i / |c_i - y_jq|^3 ]_FP64
//        - (the value the P2P kernel produces for the same points, per unit x_j),
// over the quadrature points of j that the P2P kernel visits (those in leaves
// adjacent to i's leaf).  For j = i the exact value is zero (flat panel).
// Adding D x in FP64 after the near field therefore replaces the FP32
// (or FP64) near-field values of these pairs by their FP64 quadrature.
// Exact integral over the flat triangle v[0..8] of the normal field of a unit
// density, times 4 pi:  -n . int_T (t - y) / |t - y|^3 dA_y.  The integrand
// splits into the part along the triangle's normal, which integrates to the
// solid angle the triangle subtends at t (the triple-product formula for a
// triangle's solid angle), and the in-plane part, which the divergence
// theorem in the plane turns into one logarithm per edge:
//   int_T (t - y)/R^3 dA = nu Om(t) + sum_edges m_e log((R_b + s_b)/(R_a + s_a)),
// Om > 0 when t is on the side of the unit normal nu, m_e the edge's outward
// in-plane normal, s the coordinate along the edge from the foot of t.  t
// must not lie on the triangle itself (a collocation point is never on
// another panel).
__device__ double tri_normal_field_4pi(const double t[3], const double n[3], const double *v) {
    double a[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) a[k][c] = v[3 * k + c] - t[c];  // vertices relative to t
    const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double nu[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double lnu = sqrt(nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2]);
    nu[0] /= lnu;
    nu[1] /= lnu;
    nu[2] /= lnu;
    double len[3];
    for (int k = 0; k < 3; ++k) len[k] = sqrt(a[k][0] * a[k][0] + a[k][1] * a[k][1] + a[k][2] * a[k][2]);
    const double c12[3] = {a[1][1] * a[2][2] - a[1][2] * a[2][1], a[1][2] * a[2][0] - a[1][0] * a[2][2],
                           a[1][0] * a[2][1] - a[1][1] * a[2][0]};
    const double trip = a[0][0] * c12[0] + a[0][1] * c12[1] + a[0][2] * c12[2];
    auto d3 = [](const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    const double den = len[0] * len[1] * len[2] + d3(a[0], a[1]) * len[2] + d3(a[0], a[2]) * len[1] +
                       d3(a[1], a[2]) * len[0];
    // atan2 gives half the angle seen with the vertices counter-clockwise,
    // i.e. from the side opposite to nu
    const double om = -2.0 * atan2(trip, den);
    double f[3] = {nu[0] * om, nu[1] * om, nu[2] * om};
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        double te[3] = {a[b][0] - a[e][0], a[b][1] - a[e][1], a[b][2] - a[e][2]};
        const double lt = sqrt(d3(te, te));
        te[0] /= lt;
        te[1] /= lt;
        te[2] /= lt;
        const double m[3] = {te[1] * nu[2] - te[2] * nu[1], te[2] * nu[0] - te[0] * nu[2],
                             te[0] * nu[1] - te[1] * nu[0]};
        const double sa = d3(a[e], te), sb = d3(a[b], te);
        const double lg = (sa + sb >= 0.0) ? log((len[b] + sb) / (len[e] + sa)) : log((len[e] - sa) / (len[b] - sb));
        f[0] += m[0] * lg;
        f[1] += m[1] * lg;
        f[2] += m[2] * lg;
    }
    return -d3(n, f);
}

// Near-singular candidates of collocation point i: the panels j of the
// leaves adjacent to i's leaf with |c_i - c_j| <= 2.5 sqrt(A_i).  Far
// candidates are rejected in FP32 with a relative margin of 1e-3 on the
// squared distance (far above its rounding error), the rest decided in FP64,
// so the set is exactly the FP64 rule's.  Writes the count (cnt) or, with
// off set, the columns and rows of i's entries.
__global__ void k_near_pairs(int64_t np, const int *nbr_off, const int *nbr, const int *cen_beg,
                             const double *cen64, const double *area64, const int *leaf_of_cen, const int *off,
                             int *cnt, int *col, int *row) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int T_ = leaf_of_cen[i];
    const double ci[3] = {cen64[3 * i], cen64[3 * i + 1], cen64[3 * i + 2]};
    const double tau2 = 6.25 * area64[i];
    const float cx = (float)ci[0], cy = (float)ci[1], cz = (float)ci[2];
    const float lo = (float)(tau2 * 0.999), hi = (float)(tau2 * 1.001);
    int n = 0;
    const int base = off ? off[i] : 0;
    for (int e = nbr_off[T_]; e < nbr_off[T_ + 1]; ++e) {
        const int S = nbr[e];
        for (int j = cen_beg[S]; j < cen_beg[S + 1]; ++j) {
            const float fx = cx - (float)cen64[3 * j], fy = cy - (float)cen64[3 * j + 1],
                        fz = cz - (float)cen64[3 * j + 2];
            const float f2 = fx * fx + fy * fy + fz * fz;
            if (f2 > hi) continue;
            if (f2 >= lo) {
                const double dx = ci[0] - cen64[3 * j], dy = ci[1] - cen64[3 * j + 1], dz = ci[2] - cen64[3 * j + 2];
                if (dx * dx + dy * dy + dz * dz > tau2) continue;
            }
            if (off) {
                col[base + n] = j;
                row[base + n] = (int)i;
            }
            ++n;
        }
    }
    if (!off) cnt[i] = n;
}

// 1/sqrt(x) in FP64 by Newton's iteration y <- y (3 - x y^2) / 2 from the
// FP32 hardware estimate (about 22 correct bits; two steps reach the FP64
// rounding level): cheaper on this GPU than an FP64 divide and square root.
__device__ __forceinline__ double rsqrt_newton(double x) {
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x, y * y, 1.5);
    y = y * fma(-0.5 * x, y * y, 1.5);
    return y;
}

// FP64 correction of table entry e = (i, j):
//   D_ij = 1/(4 pi) sum_q [ -A_j w_q (c_i - y_jq).n_i / |c_i - y_jq|^3 ]_FP64
//        - (the value the near-field kernel produces for the same points, per unit x_j),
// over the points of j the near-field kernel visits (those in leaves adjacent
// to i's leaf; for j = i the exact value is zero: a flat panel).  Adding D x
// after the near field replaces the FP32 (or FP64) values of these pairs by
// their FP64 quadrature.  With pan set (the exact flat-panel integrals) the
// pair's whole value, near and far points alike, becomes the exact integral.
// NQ: the rule's points (7 or 1), fixed so that their loads issue together.
template <class T, int NQ>
__global__ void k_near_values(int64_t nnz, const int *col, const int *row, const int4 *ijk, int leaf0,
                              const uint64_t *qp_key, int shift, double h, const double *cen64,
                              const double *nrm64, const double *qpg64, const double *qw64, const int *qp_of_panel,
                              const typename V4T<T>::t *trec, const typename V4T<T>::t *nrec,
                              const typename V4T<T>::t *srec, const int *leaf_of_cen, double *val,
                              const double *pan, const int *perm) {
    using V4 = typename V4T<T>::t;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = row[e], j = col[e];
    int kk[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) kk[q] = qp_of_panel[(int64_t)j * NQ + q];
    const int4 ct = ijk[leaf0 + leaf_of_cen[i]];
    const double ci[3] = {cen64[3 * i], cen64[3 * i + 1], cen64[3 * i + 2]};
    const double ni[3] = {nrm64[3 * i], nrm64[3 * i + 1], nrm64[3 * i + 2]};
    const V4 tr = trec[i], nr = nrec[i];
    auto cb = [](uint64_t v) {  // one coordinate of a Morton key
        v &= 0x1249249249249249ull;
        v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
        v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
        v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
        v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
        v = (v ^ (v >> 32)) & 0x1fffffull;
        return (int)v;
    };
    const double hT = (double)(T)h;  // the near-field kernel receives h in T
    double exact = 0.0, rep = 0.0, quad = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int k = kk[q];
        const double ex = ci[0] - qpg64[3 * k], ey = ci[1] - qpg64[3 * k + 1], ez = ci[2] - qpg64[3 * k + 2];
        double term = 0.0;
        if (j != i) {
            const double ri = rsqrt_newton(ex * ex + ey * ey + ez * ez);
            term = -qw64[k] * (ex * ni[0] + ey * ni[1] + ez * ni[2]) * (ri * ri * ri);
        }
        quad += term;
        const uint64_t kq = qp_key[k] >> shift;
        const int a = cb(kq), b = cb(kq >> 1), c = cb(kq >> 2);
        if (abs(a - ct.x) > 1 || abs(b - ct.y) > 1 || abs(c - ct.z) > 1) continue;
        exact += term;
        // replay of the near-field kernel for this point
        V4 y = srec[k];
        y.x += (T)((double)(a - ct.x) * hT);
        y.y += (T)((double)(b - ct.y) * hT);
        y.z += (T)((double)(c - ct.z) * hT);
        T nd, ri3;
        dn_pair<T>(tr.x - y.x, tr.y - y.y, tr.z - y.z, nr.x, nr.y, nr.z, nd, ri3);
        rep += -(double)y.w * (double)nd * (double)ri3;
    }
    if (pan && j != i) exact += tri_normal_field_4pi(ci, ni, pan + 9 * (int64_t)perm[j]) - quad;
    val[e] = (exact - rep) / FOUR_PI;
}

__global__ void k_leaf_of(const int *beg, int nleaf, int *leaf_of) {
    const int l = blockIdx.x;
    for (int i = beg[l] + threadIdx.x; i < beg[l + 1]; i += blockDim.x) leaf_of[i] = l;
}


// ---------------------------------------------------------------- combine
template <class T>
__global__ void k_combine(const T *far, const T *near, int64_t n, double scale, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    if (far) v += (double)far[i];
    if (near) v += (double)near[i];
    out[i] = scale * v;
}

// ---------------------------------------------------------------- tables
// Host-side FP64 solid harmonics (full m range) for the translation tables.
static void host_regular_full(double x, double y, double z, int p, std::vector<double> &out) {
    // out[(n*(2p+1) + m + p)*2 + {0,1}]
    const int W = 2 * p + 1;
    out.assign((size_t)(p + 1) * W * 2, 0.0);
    const double r2 = x * x + y * y + z * z;
    std::vector<double> re((p + 1) * (p + 1), 0.0), im((p + 1) * (p + 1), 0.0);
    auto at = [&](int n, int m) { return n * (p + 1) + m; };
    re[at(0, 0)] = 1.0;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            double f = -1.0 / (2.0 * m);
            double a = re[at(m - 1, m - 1)], b = im[at(m - 1, m - 1)];
            re[at(m, m)] = f * (x * a - y * b);
            im[at(m, m)] = f * (x * b + y * a);
        }
        if (m + 1 <= p) {
            re[at(m + 1, m)] = z * re[at(m, m)];
            im[at(m + 1, m)] = z * im[at(m, m)];
        }
        for (int n = m + 2; n <= p; ++n) {
            double c = 1.0 / ((n + m) * (double)(n - m));
            re[at(n, m)] = ((2 * n - 1) * z * re[at(n - 1, m)] - r2 * re[at(n - 2, m)]) * c;
            im[at(n, m)] = ((2 * n - 1) * z * im[at(n - 1, m)] - r2 * im[at(n - 2, m)]) * c;
        }
    }
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            int am = m < 0 ? -m : m;
            double a = re[at(n, am)], b = im[at(n, am)];
            if (m < 0) {
                double sg = (am & 1) ? -1.0 : 1.0;
                a *= sg;
                b *= -sg;
            }
            out[((size_t)n * W + m + p) * 2] = a;
            out[((size_t)n * W + m + p) * 2 + 1] = b;
        }
}

static void host_irregular_full(double x, double y, double z, int N, std::vector<double> &out) {
    // out[(n*(2N+1) + m + N)*2 + {0,1}], n <= N
    const int W = 2 * N + 1;
    out.assign((size_t)(N + 1) * W * 2, 0.0);
    const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    std::vector<double> re((N + 1) * (N + 1), 0.0), im((N + 1) * (N + 1), 0.0);
    auto at = [&](int n, int m) { return n * (N + 1) + m; };
    re[at(0, 0)] = std::sqrt(ir2);
    for (int m = 0; m <= N; ++m) {
        if (m > 0) {
            double f = -(2.0 * m - 1.0) * ir2;
            double a = re[at(m - 1, m - 1)], b = im[at(m - 1, m - 1)];
            re[at(m, m)] = f * (x * a - y * b);
            im[at(m, m)] = f * (x * b + y * a);
        }
        if (m + 1 <= N) {
            re[at(m + 1, m)] = (2.0 * m + 1.0) * z * ir2 * re[at(m, m)];
            im[at(m + 1, m)] = (2.0 * m + 1.0) * z * ir2 * im[at(m, m)];
        }
        for (int n = m + 2; n <= N; ++n) {
            double c2 = (double)(n - 1 - m) * (double)(n - 1 + m);
            re[at(n, m)] = ((2 * n - 1) * z * re[at(n - 1, m)] - c2 * re[at(n - 2, m)]) * ir2;
            im[at(n, m)] = ((2 * n - 1) * z * im[at(n - 1, m)] - c2 * im[at(n - 2, m)]) * ir2;
        }
    }
    for (int n = 0; n <= N; ++n)
        for (int m = -n; m <= n; ++m) {
            int am = m < 0 ? -m : m;
            double a = re[at(n, am)], b = im[at(n, am)];
            if (m < 0) {
                double sg = (am & 1) ? -1.0 : 1.0;
                a *= sg;
                b *= -sg;
            }
            out[((size_t)n * W + m + N) * 2] = a;
            out[((size_t)n * W + m + N) * 2 + 1] = b;
        }
}

static bool g_consts_up[64] = {};
static std::mutex g_consts_mu;

static void upload_constants(int dev) {
    std::lock_guard<std::mutex> lk(g_consts_mu);
    if (dev >= 0 && dev < 64 && g_consts_up[dev]) return;
    double rd[MAXP + 1][MAXP + 1] = {};
    float rf[MAXP + 1][MAXP + 1] = {};
    double i2d[MAXP + 1] = {};
    float i2f[MAXP + 1] = {};
    double p2d[2 * MAXP + 2];
    float p2f[2 * MAXP + 2];
    unsigned char tn[(MAXP + 1) * (MAXP + 2) / 2], tm[(MAXP + 1) * (MAXP + 2) / 2];
    for (int n = 0; n <= MAXP; ++n)
        for (int m = 0; m <= MAXP; ++m)
            if (m < n) {
                rd[n][m] = 1.0 / ((double)(n + m) * (double)(n - m));
                rf[n][m] = (float)rd[n][m];
            }
    for (int m = 1; m <= MAXP; ++m) {
        i2d[m] = 1.0 / (2.0 * m);
        i2f[m] = (float)i2d[m];
    }
    for (int j = 0; j < 2 * MAXP + 2; ++j) {
        p2d[j] = std::ldexp(1.0, -j);
        p2f[j] = (float)p2d[j];
    }
    int t = 0;
    for (int n = 0; n <= MAXP; ++n)
        for (int m = 0; m <= n; ++m) {
            tn[t] = (unsigned char)n;
            tm[t] = (unsigned char)m;
            ++t;
        }
    BEM_CUDA(cudaMemcpyToSymbol(c_rinv_d, rd, sizeof(rd)));
    BEM_CUDA(cudaMemcpyToSymbol(c_rinv_f, rf, sizeof(rf)));
    BEM_CUDA(cudaMemcpyToSymbol(c_inv2m_d, i2d, sizeof(i2d)));
    BEM_CUDA(cudaMemcpyToSymbol(c_inv2m_f, i2f, sizeof(i2f)));
    BEM_CUDA(cudaMemcpyToSymbol(c_pow2n_d, p2d, sizeof(p2d)));
    BEM_CUDA(cudaMemcpyToSymbol(c_pow2n_f, p2f, sizeof(p2f)));
    BEM_CUDA(cudaMemcpyToSymbol(c_tri_n, tn, sizeof(tn)));
    BEM_CUDA(cudaMemcpyToSymbol(c_tri_m, tm, sizeof(tm)));
    if (dev >= 0 && dev < 64) g_consts_up[dev] = true;
}

// Real (p+1)^2 x (p+1)^2 matrix of a complex translation
//   out_k^l = sum_{n, m=-n..n} coef(k, l, n, m) in_n^m
// acting on the compact real layout (both sides real fields, so
// in_n^{-m} = (-1)^m conj(in_n^m)).  With P = coef(k,l,n,mu) and
// Q = (-1)^mu coef(k,l,n,-mu), an input a + ib at (n, mu) contributes
// a (P + Q) + i b (P - Q).  Stored column-major: Tt[in * nc + out].
template <class F>
static void real_operator(int p, F coef, double *Tt) {
    const int nc = (p + 1) * (p + 1);
    std::fill(Tt, Tt + (size_t)nc * nc, 0.0);
    for (int k = 0; k <= p; ++k)
        for (int l = 0; l <= k; ++l) {
            const int ro = k * k + (l == 0 ? 0 : 2 * l - 1), io = l > 0 ? k * k + 2 * l : -1;
            for (int n = 0; n <= p; ++n)
                for (int mu = 0; mu <= n; ++mu) {
                    double Pr, Pi, Qr = 0, Qi = 0;
                    coef(k, l, n, mu, Pr, Pi);
                    if (mu > 0) {
                        coef(k, l, n, -mu, Qr, Qi);
                        if (mu & 1) { Qr = -Qr; Qi = -Qi; }
                    }
                    const int ri = n * n + (mu == 0 ? 0 : 2 * mu - 1), ii = mu > 0 ? n * n + 2 * mu : -1;
                    Tt[(size_t)ri * nc + ro] += Pr + Qr;
                    if (ii >= 0) Tt[(size_t)ii * nc + ro] += -(Pi - Qi);
                    if (io >= 0) Tt[(size_t)ri * nc + io] += Pi + Qi;
                    if (io >= 0 && ii >= 0) Tt[(size_t)ii * nc + io] += Pr - Qr;
                }
        }
}

void ensure_smem_attr(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    BEM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = done[{func, dev}];
    if (bytes <= cur) return;
    BEM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

struct TabKey {
    int dev, p, prec, ws;
    bool operator<(const TabKey &o) const {
        if (dev != o.dev) return dev < o.dev;
        if (p != o.p) return p < o.p;
        if (prec != o.prec) return prec < o.prec;
        return ws < o.ws;
    }
};
static std::mutex g_tab_mu;
static std::map<TabKey, std::weak_ptr<Tables>> g_tab_cache;

template <class T>
static void upload(DArray<T> &d, const std::vector<double> &h) {
    std::vector<T> v(h.begin(), h.end());
    d.alloc(v.size());
    BEM_CUDA(cudaMemcpy(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

static std::shared_ptr<Tables> make_tables(int p, int prec, int ws) {
    auto t = std::make_shared<Tables>();
    const int W = 2 * p + 1, W2 = 4 * p + 1;
    const int nc = (p + 1) * (p + 1);
    const int NOFFSET = m2l_classes(ws), RO = m2l_radius(ws), WO = 2 * RO + 1;
    t->p = p;
    t->ws = ws;
    // parent/child offsets: child centre minus parent centre over the parent size
    std::vector<std::vector<double>> r8(8);
    std::vector<double> rtab((size_t)8 * (p + 1) * W * 2);
    for (int o = 0; o < 8; ++o) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = ((o >> k) & 1) ? 0.25 : -0.25;
        host_regular_full(d[0], d[1], d[2], p, r8[o]);
        std::memcpy(&rtab[(size_t)o * (p + 1) * W * 2], r8[o].data(), r8[o].size() * sizeof(double));
    }
    // M2L offsets: target centre minus source centre over the cell size = -(dx,dy,dz)
    const size_t itot = (size_t)(2 * p + 1) * W2 * 2;
    std::vector<double> it((size_t)NOFFSET * itot, 0.0), tmp;
    auto offset_of = [&](int o, int &dx, int &dy, int &dz) {
        dx = o / (WO * WO) - RO;
        dy = (o / WO) % WO - RO;
        dz = o % WO - RO;
        return std::abs(dx) > ws || std::abs(dy) > ws || std::abs(dz) > ws;  // a class in use
    };
    for (int o = 0; o < NOFFSET; ++o) {
        int dx, dy, dz;
        if (!offset_of(o, dx, dy, dz)) continue;
        host_irregular_full(-dx, -dy, -dz, 2 * p, tmp);
        std::memcpy(&it[(size_t)o * itot], tmp.data(), tmp.size() * sizeof(double));
    }
    // dense real operators
    const size_t osz = (size_t)nc * nc;
    std::vector<double> om2l((size_t)NOFFSET * osz, 0.0), om2m(8 * osz), ol2l(8 * osz);
    for (int o = 0; o < NOFFSET; ++o) {
        int dx, dy, dz;
        if (!offset_of(o, dx, dy, dz)) continue;
        const double *I = &it[(size_t)o * itot];
        // L_k^l = (-1)^k sum M_n^m I_{n+k}^{m+l}
        real_operator(p, [&](int k, int l, int n, int m, double &re, double &im) {
            const double sg = (k & 1) ? -1.0 : 1.0;
            const size_t q = ((size_t)(n + k) * W2 + (m + l) + 2 * p) * 2;
            re = sg * I[q];
            im = sg * I[q + 1];
        }, &om2l[(size_t)o * osz]);
    }
    for (int o = 0; o < 8; ++o) {
        const std::vector<double> &R = r8[o];
        auto Rc = [&](int n, int m, double &re, double &im) {  // conj(R_n^m), 0 outside
            if (n < 0 || m < -n || m > n) { re = im = 0; return; }
            const size_t q = ((size_t)n * W + m + p) * 2;
            re = R[q];
            im = -R[q + 1];
        };
        // M2M: M'_N^Mo = sum_{j,mu} 2^-j conj(R_{N-j}^{Mo-mu}) M_j^mu
        real_operator(p, [&](int N, int Mo, int j, int mu, double &re, double &im) {
            if (j > N) { re = im = 0; return; }
            Rc(N - j, Mo - mu, re, im);
            const double s = std::ldexp(1.0, -j);
            re *= s;
            im *= s;
        }, &om2m[(size_t)o * osz]);
        // L2L: L'_k^l = 2^-(k+1) sum_{n,m} conj(R_{n-k}^{m-l}) L_n^m
        real_operator(p, [&](int k, int l, int n, int m, double &re, double &im) {
            if (n < k) { re = im = 0; return; }
            Rc(n - k, m - l, re, im);
            const double s = std::ldexp(1.0, -(k + 1));
            re *= s;
            im *= s;
        }, &ol2l[(size_t)o * osz]);
    }
    if (prec == BEM_MIXED && nc <= 128) {
        std::vector<float> op;
        build_tc_tables(p, om2l, NOFFSET, op);
        t->Tc_f.alloc(op.size());
        BEM_CUDA(cudaMemcpy(t->Tc_f.p, op.data(), op.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    // translation operators with each [in] row padded to the cell stride, so
    // that k_translate stages them with 16-byte copies
    const int ld = cell_stride(p);
    auto pad = [&](const std::vector<double> &ops, int nops) {
        std::vector<double> r((size_t)nops * nc * ld, 0.0);
        for (size_t o = 0; o < (size_t)nops; ++o)
            for (int k = 0; k < nc; ++k)
                std::copy_n(&ops[(o * nc + k) * nc], nc, &r[(o * nc + k) * ld]);
        return r;
    };
    const std::vector<double> pm2l = pad(om2l, NOFFSET), pm2m = pad(om2m, 8), pl2l = pad(ol2l, 8);
    if (prec == BEM_MIXED) {
        upload(t->Rm2m_f, rtab);
        upload(t->If_f, it);
        upload(t->Om2l_f, pm2l);
        upload(t->Om2m_f, pm2m);
        upload(t->Ol2l_f, pl2l);
    } else {
        upload(t->Rm2m_d, rtab);
        upload(t->If_d, it);
        upload(t->Om2l_d, pm2l);
        upload(t->Om2m_d, pm2m);
        upload(t->Ol2l_d, pl2l);
    }
    return t;
}

static std::shared_ptr<Tables> cached_tables(int dev, int p, int prec, int ws) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    TabKey key{dev, p, prec, ws};
    auto it = g_tab_cache.find(key);
    if (it != g_tab_cache.end())
        if (auto sp = it->second.lock()) return sp;
    auto t = make_tables(p, prec, ws);
    g_tab_cache[key] = t;
    return t;
}

// The panel tree's tables (one-cell separation) and, when the charge tree is
// separated by two cells, its own set.
void build_tables(Mesh &m) {
    upload_constants(m.device);
    m.tab = cached_tables(m.device, m.opt.p, m.opt.precision, 1);
    if (m.tc.ws == 2) m.tab2 = cached_tables(m.device, m.opt.p, m.opt.precision, 2);
    else m.tab2.reset();
}

const Tables &tables_for(const Mesh &m, const Tree &t) {
    const Tables *tb = t.ws == 2 ? m.tab2.get() : m.tab.get();
    if (!tb || tb->ws != t.ws) throw Error(BEM_ECUDA, "translation tables missing for the tree's separation");
    return *tb;
}

// ------------------------------------------------- batched dense translations
// out[pair_out[j]] += Op[op] . in[pair_in[j]] for the pairs of one chunk: a
// (p+1)^2 x (p+1)^2 by (p+1)^2 x 64 product tiled 128 x 64 x BK through
// shared memory, 8 x 4 outputs per thread, then scattered with coalesced
// atomic adds (a warp adds 32 consecutive coefficients of one cell).
constexpr int TR_BM = 128, TR_THREADS = 256;
constexpr int TR_THREADS_TREE = 256;  // M2M / L2L kernels (chunks of TR_BN_TREE pairs)
constexpr int TR_BN_M2L = 64;  // pairs per chunk for M2L (many pairs per offset class)
constexpr int TR_BN_TREE = 32; // pairs per chunk for M2M / L2L (8 operators per level)
template <class T> struct TrBK;
template <> struct TrBK<float> { static constexpr int v = 32; };
template <> struct TrBK<double> { static constexpr int v = 16; };

constexpr int TR_NS = 4;  // cp.async stages of the K loop (p <= 10 fits in one round)

// One element copied global -> shared without passing through registers;
// ok = false writes zero (src-size 0: nothing is read).
template <class T>
__device__ __forceinline__ void cp_async_elt(T *dst, const T *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = ok ? (int)sizeof(T) : 0;
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// out[p_out[j]] += Op[class] x in[p_in[j]] for the pairs of one chunk (one
// operator class): a [BM x nc] x [nc x BN] product whose K loop is staged
// through TR_NS shared-memory buffers by cp.async (the operator rows, padded
// to the cell stride, in 16-byte copies), so every tile's loads are in flight
// together.  NTH threads; each owns 8 consecutive output rows (two or four
// 16-byte shared loads per k) and BN x 16 / NTH pair columns.
template <class T, int BN, int NTH>
__global__ void __launch_bounds__(NTH)
k_translate(const T *__restrict__ ops, int nc, int cs, const int4 *__restrict__ chunks,
            const int *__restrict__ p_out, const int *__restrict__ p_in, const T *__restrict__ in,
            T *__restrict__ out) {
    constexpr int BK = TrBK<T>::v;
    constexpr int NTY = TR_BM / 8;          // row groups of 8
    constexpr int NTX = NTH / NTY;          // column groups
    constexpr int CPT = BN / NTX;           // columns per thread
    static_assert(NTH % NTY == 0 && BN % NTX == 0, "translate tiling");
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int STAGE = BK * TR_BM + BK * BN;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);   // TR_NS x {As [BK][BM], Bs [BK][BN]}
    T *Cs = sm;                             // [BN][BM+1] (epilogue)
    __shared__ int s_in[BN], s_out[BN];
    const int4 ch = chunks[blockIdx.x];
    const T *Tt = ops + (size_t)ch.x * nc * cs;
    const int rb = blockIdx.y * TR_BM;
    const int tid = threadIdx.x, ty = tid / NTX, tx = tid - ty * NTX;
    if (tid < BN) {
        s_in[tid] = tid < ch.z ? p_in[ch.y + tid] : -1;
        s_out[tid] = tid < ch.z ? p_out[ch.y + tid] : -1;
    }
    T acc[8][CPT];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[r][c] = 0;
    __syncthreads();
    const int nk = (nc + BK - 1) / BK;
    auto issue = [&](int kt) {
        T *As = sm + (kt % TR_NS) * STAGE;
        T *Bs = As + BK * TR_BM;
        const int k0 = kt * BK;
        for (int e = tid; e < BK * TR_BM / VEC; e += NTH) {
            const int k = e / (TR_BM / VEC), r = (e - k * (TR_BM / VEC)) * VEC;
            const bool ok = k0 + k < nc && rb + r < cs;  // cs % VEC == 0: a copy never crosses a row
            cp_async_16(As + k * TR_BM + r, ok ? Tt + (size_t)(k0 + k) * cs + rb + r : Tt, ok);
        }
        for (int e = tid; e < BK * BN; e += NTH) {
            const int k = e / BN, j = e - k * BN;
            const int src = s_in[j];
            const bool ok = src >= 0 && k0 + k < nc;
            cp_async_elt(Bs + e, ok ? in + (size_t)src * cs + k0 + k : in, ok);
        }
    };
#pragma unroll
    for (int st = 0; st < TR_NS - 1; ++st) {
        if (st < nk) issue(st);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<TR_NS - 2>();  // this thread's copies of tile kt have landed
        __syncthreads();             // everyone's have; stage (kt - 1) % TR_NS is free again
        if (kt + TR_NS - 1 < nk) issue(kt + TR_NS - 1);
        cp_async_commit();
        const T *As = sm + (kt % TR_NS) * STAGE;
        const T *Bs = As + BK * TR_BM;
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            T a[8], b[CPT];
#pragma unroll
            for (int q = 0; q < 8; q += VEC) {
                if constexpr (sizeof(T) == 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(As + k * TR_BM + ty * 8 + q);
                    a[q] = v.x;
                    a[q + 1] = v.y;
                    a[q + 2] = v.z;
                    a[q + 3] = v.w;
                } else {
                    const double2 v = *reinterpret_cast<const double2 *>(As + k * TR_BM + ty * 8 + q);
                    a[q] = v.x;
                    a[q + 1] = v.y;
                }
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) b[c] = Bs[k * BN + tx * CPT + c];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < CPT; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) Cs[(tx * CPT + c) * (TR_BM + 1) + ty * 8 + r] = acc[r][c];
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int rows = min(TR_BM, nc - rb);
    for (int j = warp; j < ch.z; j += NTH / 32) {
        T *o = out + (size_t)s_out[j] * cs + rb;
        const T *cj = Cs + j * (TR_BM + 1);
        for (int r = lane; r < rows; r += 32) atomicAdd(o + r, cj[r]);
    }
}

// M2M / L2L: out[p_out[j]] += Op[octant] . in[p_in[j]] for a chunk of up to
// BN pairs of one operator.  The level's few thousand translations are
// latency-bound, so the CTA copies the whole operator block (nc x TR_BM) and
// the chunk's BN input rows to shared memory in one round of 16-byte
// cp.async, then each thread forms 8 rows x (BN / 16) pair columns (columns
// strided by 16; input rows padded to 4 mod 32 words: at most 2-way bank
// conflicts) and the results leave as coalesced atomic adds.
template <class T, int BN, int NTH, int BM>
__device__ __forceinline__ void tree_translate_block(const T *__restrict__ ops, int nc, int cs, int ldb, int4 ch,
                                                     int rb, const int *__restrict__ p_out,
                                                     const int *__restrict__ p_in, const T *__restrict__ in,
                                                     T *__restrict__ out, unsigned char *smraw, int *s_in,
                                                     int *s_out) {
    constexpr int TR_BM = BM;       // output rows of this CTA
    constexpr int NTY = TR_BM / 8;  // row groups of 8
    constexpr int NTX = NTH / NTY;  // column groups
    constexpr int CPT = BN / NTX;   // columns per thread
    static_assert(NTH % NTY == 0 && BN % NTX == 0, "tree translate tiling");
    constexpr int VEC = 16 / (int)sizeof(T);
    T *As = reinterpret_cast<T *>(smraw);  // [nc][TR_BM]
    T *Bs = As + (size_t)nc * TR_BM;       // [BN][ldb]
    T *Cs = As;                            // [BN][TR_BM + 1] (epilogue)
    const T *Tt = ops + (size_t)ch.x * nc * cs;
    // a warp covers 8 pair columns x 4 row groups: its input-row loads hit 8
    // different banks and its operator loads one 128-byte span
    static_assert(NTX % 8 == 0, "tree translate thread map");
    const int tid = threadIdx.x, rest = tid >> 3, ty = rest % NTY, tx = (tid & 7) + 8 * (rest / NTY);
    // The next level's launch may start now (programmatic dependent launch):
    // its operator rows and pair lists do not depend on this level.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid < BN) {
        s_in[tid] = tid < ch.z ? p_in[ch.y + tid] : -1;
        s_out[tid] = tid < ch.z ? p_out[ch.y + tid] : -1;
    }
    __syncthreads();
    for (int e = tid; e < nc * (TR_BM / VEC); e += NTH) {
        const int k = e / (TR_BM / VEC), r = (e - k * (TR_BM / VEC)) * VEC;
        const bool ok = rb + r < cs;  // cs % VEC == 0: a copy never crosses a row
        cp_async_16(As + (size_t)k * TR_BM + r, ok ? Tt + (size_t)k * cs + rb + r : Tt, ok);
    }
    // everything the previous kernels of the stream wrote (this level's input
    // expansions, the cleared outputs) is complete and visible after this
    // wait; nothing above reads or writes it
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int cv = cs / VEC;
    for (int e = tid; e < BN * cv; e += NTH) {
        const int j = e / cv, q = (e - j * cv) * VEC;
        const int src = s_in[j];
        cp_async_16(Bs + (size_t)j * ldb + q, src >= 0 ? in + (size_t)src * cs + q : in, src >= 0);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    T acc[8][CPT];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[r][c] = 0;
#pragma unroll 4
    for (int k = 0; k < nc; ++k) {
        T a[8], b[CPT];
#pragma unroll
        for (int q = 0; q < 8; q += VEC) {
            if constexpr (sizeof(T) == 4) {
                const float4 v = *reinterpret_cast<const float4 *>(As + (size_t)k * TR_BM + ty * 8 + q);
                a[q] = v.x;
                a[q + 1] = v.y;
                a[q + 2] = v.z;
                a[q + 3] = v.w;
            } else {
                const double2 v = *reinterpret_cast<const double2 *>(As + (size_t)k * TR_BM + ty * 8 + q);
                a[q] = v.x;
                a[q + 1] = v.y;
            }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) b[c] = Bs[(size_t)(tx + NTX * c) * ldb + k];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) Cs[(tx + NTX * c) * (TR_BM + 1) + ty * 8 + r] = acc[r][c];
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int rows = min(TR_BM, nc - rb);
    for (int j = warp; j < ch.z; j += NTH / 32) {
        T *o = out + (size_t)s_out[j] * cs + rb;
        const T *cj = Cs + j * (TR_BM + 1);
        for (int r = lane; r < rows; r += 32) atomicAdd(o + r, cj[r]);
    }
}

template <class T, int BN, int NTH, int BM>
__global__ void __launch_bounds__(NTH)
k_tree_translate(const T *__restrict__ ops, int nc, int cs, int ldb, const int4 *__restrict__ chunks,
                 const int *__restrict__ p_out, const int *__restrict__ p_in, const T *__restrict__ in,
                 T *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_in[BN], s_out[BN];
    tree_translate_block<T, BN, NTH, BM>(ops, nc, cs, ldb, chunks[blockIdx.x], blockIdx.y * BM, p_out, p_in, in, out,
                                         smraw, s_in, s_out);
}

// input-row pitch of k_tree_translate (4 mod 32 words) and its shared memory
template <class T>
static int tree_ldb(int cs) {
    return (int)(((cs * sizeof(T) + 127) / 128 * 128 + 16) / sizeof(T));
}
constexpr int TREE_BM = 64;  // operator rows per CTA (two CTAs per chunk at p = 10)
template <class T>
static size_t tree_translate_smem(int nc, int cs) {
    const size_t ab = ((size_t)nc * TREE_BM + (size_t)TR_BN_TREE * tree_ldb<T>(cs)) * sizeof(T);
    return std::max(ab, (size_t)TR_BN_TREE * (TREE_BM + 1) * sizeof(T));
}
constexpr size_t TREE_SMEM_MAX = 200 * 1024;  // above: the pipelined k_translate

template <class T, int BN>
static size_t translate_smem() {
    constexpr int BK = TrBK<T>::v;
    const size_t a = (size_t)TR_NS * (BK * TR_BM + BK * BN) * sizeof(T);
    const size_t c = (size_t)BN * (TR_BM + 1) * sizeof(T);
    return std::max(a, c);
}

__global__ void k_iota(int *a, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int)i;
}

__global__ void k_class_count(const int *key, int64_t n, int *cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(cnt + key[i], 1);
}

// grouped pair d is list entry e = perm[d]
__global__ void k_gather_pairs(const int *perm, const int *po, const int *pi, int64_t n, int *g_out, int *g_in) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= n) return;
    const int e = perm[d];
    g_out[d] = po[e];
    g_in[d] = pi[e];
}


// Group the translations of a tree by operator and cut them into chunks.
__global__ void k_m2l_pairs(const int *m2l_off, int first, int last, const int *m2l_src,
                            const int *m2l_ofs, int *out, int *in, int *key) {
    const int t = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= last) return;
    for (int e = m2l_off[t]; e < m2l_off[t + 1]; ++e) {
        out[e] = t;
        in[e] = m2l_src[e];
        key[e] = m2l_ofs[e];
    }
}

// Launch order of the near-field kernel: leaves by decreasing work
// (targets x sources of the adjacent leaves), so that the last wave of
// CTAs holds the small ones.
static void build_p2p_order(Mesh &m, Tree &t) {
    cudaStream_t s = m.stream;
    const int n = t.nleaf;
    std::vector<int> tb(n + 1), qb(n + 1), cb(n + 1), no(n + 1), nb(t.nnbr > 0 ? t.nnbr : 1);
    BEM_CUDA(cudaMemcpyAsync(tb.data(), t.cen_beg.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(qb.data(), t.qp_beg.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(cb.data(), t.chg_beg.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(no.data(), t.nbr_off.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (t.nnbr > 0)
        BEM_CUDA(cudaMemcpyAsync(nb.data(), t.nbr.p, t.nnbr * sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<int64_t, int>> w(n);
    for (int l = 0; l < n; ++l) {
        int64_t src = 0;
        for (int e = no[l]; e < no[l + 1]; ++e) {
            const int S = nb[e];
            src += (qb[S + 1] - qb[S]) + (cb[S + 1] - cb[S]);
        }
        const int64_t tg = (tb[l + 1] - tb[l]) + (cb[l + 1] - cb[l]);
        w[l] = {-(tg * src), l};
    }
    std::stable_sort(w.begin(), w.end());
    std::vector<int> ord(n);
    for (int l = 0; l < n; ++l) ord[l] = w[l].second;
    t.p2p_order.alloc(n);
    BEM_CUDA(cudaMemcpyAsync(t.p2p_order.p, ord.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    // the near field's work lists (pair counts below 2^22 per leaf: the
    // records keep them in 23 bits)
    int maxn = 0;
    for (int l = 0; l < n; ++l) maxn = std::max(maxn, no[l + 1] - no[l]);
    for (int l = 0; l < n; ++l) {
        int64_t src = 0;
        for (int e = no[l]; e < no[l + 1]; ++e) src += std::max(qb[nb[e] + 1] - qb[nb[e]], cb[nb[e] + 1] - cb[nb[e]]);
        if (src / 2 + maxn >= (1 << 22)) throw Error(BEM_EUNSUPPORTED, "near field: too many sources next to one leaf");
    }
    if (t.ws != 1 && t.ws != 2) throw Error(BEM_EUNSUPPORTED, "near field: separation not built");
    t.p2p_nb = t.ws == 1 ? 27 : 125;
    if (maxn > t.p2p_nb) throw Error(BEM_ECUDA, "near field: neighbour list longer than the separation allows");
    std::vector<int64_t> first(n + 1, 0);
    for (int b = 0; b < n; ++b) first[b + 1] = first[b] + (t.ws == 1 ? 27 : no[ord[b] + 1] - no[ord[b]]);
    if (first[n] >= ((int64_t)1 << 31)) throw Error(BEM_EUNSUPPORTED, "near field: work list too long");
    DArray<int64_t> d_first;
    d_first.alloc(n + 1);
    BEM_CUDA(cudaMemcpyAsync(d_first.p, first.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const TreeView tv = view(t);
    const bool has[2] = {t.has_qp, t.has_chg};
    for (int k = 0; k < 2; ++k) {
        t.p2p_hdr[k] = DArray<int4>();
        t.p2p_rec[k] = DArray<int2>();
        if (!has[k] || n == 0) continue;
        t.p2p_hdr[k].alloc((size_t)3 * n);
        t.p2p_rec[k].alloc((size_t)first[n]);
        BEM_CUDA(cudaMemsetAsync(t.p2p_rec[k].p, 0, (size_t)first[n] * sizeof(int2), s));
        if (k == 0) k_p2p_list<SRC_QUAD><<<n, 128, 0, s>>>(tv, d_first.p, t.p2p_hdr[k].p, t.p2p_rec[k].p);
        else k_p2p_list<SRC_CHARGE><<<n, 128, 0, s>>>(tv, d_first.p, t.p2p_hdr[k].p, t.p2p_rec[k].p);
        BEM_CHECK_LAUNCH();
    }
    BEM_CUDA(cudaStreamSynchronize(s));
}

void build_translation_groups(Mesh &m, Tree &t) {
    cudaStream_t s = m.stream;
    const int L = t.L;
    build_p2p_order(m, t);
    t.m2m_chunk0.assign(L + 2, 0);
    t.m2m_nchunk.assign(L + 2, 0);
    t.l2l_chunk0.assign(L + 2, 0);
    t.l2l_nchunk.assign(L + 2, 0);
    t.m2l_chunk0 = t.m2l_nchunk = 0;
    if (L < 2) return;
    // host copies of the cell structure (parents, coordinates)
    std::vector<int4> ijk(t.ncell);
    std::vector<int> parent(t.ncell);
    BEM_CUDA(cudaMemcpyAsync(ijk.data(), t.ijk.p, t.ncell * sizeof(int4), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(parent.data(), t.parent.p, t.ncell * sizeof(int), cudaMemcpyDeviceToHost, s));
    // M2L pairs grouped by offset class on the device: a stable radix sort of
    // the pair indices (target-major list order) by class, the pairs gathered
    // into that order, and only the per-class counts copied to the host to cut
    // the classes into chunks
    const int64_t nm = t.nm2l;
    const int ncls = m2l_classes(t.ws);
    int cls_bits = 0;
    while ((1 << cls_bits) < ncls) ++cls_bits;
    std::vector<int4> chunks;
    std::vector<int> cnt(ncls, 0);
    const int first = t.lvl_off[2], last = t.ncell;
    if (nm > 0) {
        DArray<int> po, pi, key, idx, key_s, perm, dcnt;
        po.alloc(nm);
        pi.alloc(nm);
        key.alloc(nm);
        idx.alloc(nm);
        key_s.alloc(nm);
        perm.alloc(nm);
        dcnt.alloc(ncls);
        k_m2l_pairs<<<cdiv(last - first, 256), 256, 0, s>>>(t.m2l_off.p, first, last, t.m2l_src.p,
                                                          t.m2l_ofs.p, po.p, pi.p, key.p);
        BEM_CHECK_LAUNCH();
        k_iota<<<cdiv(nm, 256), 256, 0, s>>>(idx.p, nm);
        BEM_CHECK_LAUNCH();
        sort_pairs_int(key.p, idx.p, key_s.p, perm.p, nm, cls_bits, s);
        BEM_CUDA(cudaMemsetAsync(dcnt.p, 0, ncls * sizeof(int), s));
        k_class_count<<<cdiv(nm, 256), 256, 0, s>>>(key.p, nm, dcnt.p);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaMemcpyAsync(cnt.data(), dcnt.p, ncls * sizeof(int), cudaMemcpyDeviceToHost, s));
        // the M2L part of the grouped arrays (the tree translations are appended below)
        t.g_out.alloc(nm);
        t.g_in.alloc(nm);
        k_gather_pairs<<<cdiv(nm, 256), 256, 0, s>>>(perm.p, po.p, pi.p, nm, t.g_out.p, t.g_in.p);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> start(ncls + 1, 0);
        for (int o = 0; o < ncls; ++o) start[o + 1] = start[o] + cnt[o];
        for (int o = 0; o < ncls; ++o)
            for (int64_t b = start[o]; b < start[o + 1]; b += TR_BN_M2L)
                chunks.push_back(make_int4(o, (int)b, (int)std::min<int64_t>(TR_BN_M2L, start[o + 1] - b), 0));
    }
    t.m2l_nchunk = (int)chunks.size();
    build_tc_super(t, chunks, s);
    // M2M (out parent, in child) and L2L (out child, in parent) per child level
    std::vector<int> h_out, h_in;
    for (int c = 3; c <= L; ++c) {
        std::vector<std::vector<int>> byoct(8);
        for (int e = t.lvl_off[c]; e < t.lvl_off[c + 1]; ++e) {
            const int4 q = ijk[e];
            byoct[(q.x & 1) | ((q.y & 1) << 1) | ((q.z & 1) << 2)].push_back(e);
        }
        for (int pass = 0; pass < 2; ++pass) {
            const int c0 = (int)chunks.size();
            for (int o = 0; o < 8; ++o) {
                const int64_t b0 = nm + (int64_t)h_out.size();
                for (int e : byoct[o]) {
                    if (pass == 0) { h_out.push_back(parent[e]); h_in.push_back(e); }
                    else { h_out.push_back(e); h_in.push_back(parent[e]); }
                }
                const int64_t b1 = nm + (int64_t)h_out.size();
                for (int64_t b = b0; b < b1; b += TR_BN_TREE)
                    chunks.push_back(make_int4(o, (int)b, (int)std::min<int64_t>(TR_BN_TREE, b1 - b), 0));
            }
            if (pass == 0) { t.m2m_chunk0[c] = c0; t.m2m_nchunk[c] = (int)chunks.size() - c0; }
            else { t.l2l_chunk0[c] = c0; t.l2l_nchunk[c] = (int)chunks.size() - c0; }
        }
    }
    {
        const size_t ntot = (size_t)nm + h_out.size();
        DArray<int> go, gi;
        go.alloc(ntot);
        gi.alloc(ntot);
        if (nm > 0) {
            BEM_CUDA(cudaMemcpyAsync(go.p, t.g_out.p, nm * sizeof(int), cudaMemcpyDeviceToDevice, s));
            BEM_CUDA(cudaMemcpyAsync(gi.p, t.g_in.p, nm * sizeof(int), cudaMemcpyDeviceToDevice, s));
        }
        if (!h_out.empty()) {
            BEM_CUDA(cudaMemcpyAsync(go.p + nm, h_out.data(), h_out.size() * sizeof(int), cudaMemcpyHostToDevice, s));
            BEM_CUDA(cudaMemcpyAsync(gi.p + nm, h_in.data(), h_in.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        }
        BEM_CUDA(cudaStreamSynchronize(s));
        t.g_out = std::move(go);
        t.g_in = std::move(gi);
    }
    t.g_chunk.alloc(chunks.size());
    BEM_CUDA(cudaMemcpyAsync(t.g_chunk.p, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- driver
template <class T>
struct PassBufs;
template <>
struct PassBufs<float> {
    static float *M(Mesh &m) { return m.Mf.p; }
    static float *L(Mesh &m) { return m.Lf.p; }
    static float *far(Mesh &m) { return m.far_f.p; }
    static float *near(Mesh &m) { return m.near_f.p; }
    static const cpx<float> *R(const Tables &t) { return reinterpret_cast<const cpx<float> *>(t.Rm2m_f.p); }
    static const cpx<float> *I(const Tables &t) { return reinterpret_cast<const cpx<float> *>(t.If_f.p); }
    static const float *Om2l(const Tables &t) { return t.Om2l_f.p; }
    static const float *Om2m(const Tables &t) { return t.Om2m_f.p; }
    static const float *Ol2l(const Tables &t) { return t.Ol2l_f.p; }
    static const float4 *cen(Mesh &m) { return m.cen32.p; }
    static const float4 *nrm(Mesh &m) { return m.nrm32.p; }
    static const float4 *nrmq(Mesh &m) { return m.nrmq32.p; }
    static const float4 *qp(Mesh &m) { return m.qp32.p; }
    static const float4 *chg(Mesh &m) { return m.chg32.p; }
    static float4 *str(Mesh &m) { return m.str32.p; }
};
template <>
struct PassBufs<double> {
    static double *M(Mesh &m) { return m.Md.p; }
    static double *L(Mesh &m) { return m.Ld.p; }
    static double *far(Mesh &m) { return m.far_d.p; }
    static double *near(Mesh &m) { return m.near_d.p; }
    static const cpx<double> *R(const Tables &t) { return reinterpret_cast<const cpx<double> *>(t.Rm2m_d.p); }
    static const cpx<double> *I(const Tables &t) { return reinterpret_cast<const cpx<double> *>(t.If_d.p); }
    static const double *Om2l(const Tables &t) { return t.Om2l_d.p; }
    static const double *Om2m(const Tables &t) { return t.Om2m_d.p; }
    static const double *Ol2l(const Tables &t) { return t.Ol2l_d.p; }
    static const double4 *cen(Mesh &m) { return m.cen64r.p; }
    static const double4 *nrm(Mesh &m) { return m.nrm64r.p; }
    static const double4 *nrmq(Mesh &m) { return m.nrmq64r.p; }
    static const double4 *qp(Mesh &m) { return m.qp64r.p; }
    static const double4 *chg(Mesh &m) { return m.chg64r.p; }
    static double4 *str(Mesh &m) { return m.str64.p; }
};

// one warp per 32 targets of an average leaf, 1..4 warps
static int l2p_threads(int64_t ntgt, int nleaf) {
    const int64_t avg = nleaf > 0 ? (ntgt + nleaf - 1) / nleaf : 1;
    return (int)std::min<int64_t>(128, std::max<int64_t>(32, (avg + 31) / 32 * 32));
}

static int p2m_threads(int p, size_t elt) {
    const size_t nc = (size_t)(p + 1) * (p + 1);
    int t = 128;
    while (t > 32 && (size_t)t * nc * elt > 96 * 1024) t >>= 1;
    return t;
}

template <class T, class KernelT>
static void set_smem(KernelT kern, size_t bytes) {
    if (bytes > 48 * 1024) ensure_smem_attr(reinterpret_cast<const void *>(kern), bytes);
}


static void ev_rec(Mesh &m, bool timed, int k) {
    if (timed && m.tm.on) BEM_CUDA(cudaEventRecord(m.tm.ev[k], m.stream));
}

// one level of M2M or L2L: the chunks [chunk0, chunk0 + nchunk) of the
// grouped tree translations
template <class T>
static void tree_translate(const T *ops, int nc, int cs, int rblocks, const Tree &t, int chunk0, int nchunk,
                           const T *in, T *out, cudaStream_t s) {
    if (nchunk == 0) return;
    dim3 g(nchunk, rblocks);
    const size_t sm = tree_translate_smem<T>(nc, cs);
    if (sm <= TREE_SMEM_MAX) {
        dim3 gt(nchunk, cdiv(nc, TREE_BM));
        auto kern = k_tree_translate<T, TR_BN_TREE, TR_THREADS_TREE, TREE_BM>;
        set_smem<T>(kern, sm);
        // programmatic dependent launch: the CTAs may start while the previous
        // kernel of the stream finishes (the kernel waits before it reads its
        // input or writes its output)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = gt;
        cfg.blockDim = dim3(TR_THREADS_TREE);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const int ldb = tree_ldb<T>(cs);
        const int4 *chunks = t.g_chunk.p + chunk0;
        const int *po = t.g_out.p, *pi = t.g_in.p;
        BEM_CUDA(cudaLaunchKernelEx(&cfg, kern, ops, nc, cs, ldb, chunks, po, pi, in, out));
    } else {
        const size_t trsm_t = translate_smem<T, TR_BN_TREE>();
        set_smem<T>(k_translate<T, TR_BN_TREE, TR_THREADS_TREE>, trsm_t);
        k_translate<T, TR_BN_TREE, TR_THREADS_TREE><<<g, TR_THREADS_TREE, trsm_t, s>>>(
            ops, nc, cs, t.g_chunk.p + chunk0, t.g_out.p, t.g_in.p, in, out);
    }
    BEM_CHECK_LAUNCH();
}

// One sweep of tree translations: M2M over the child levels L .. 3, or L2L
// over 3 .. L, one launch per level.  (Measured: one launch for all levels,
// with CTAs taking items in level order and waiting on per-level counters,
// took 55 instead of 38 us for the M2M sweep of the 81,920-panel molecule:
// a level's time is its items' own latency, not the launch gaps.)
template <class T>
static void tree_sweep(Mesh &m, const T *ops, int nc, int cs, const Tree &t, bool up, const T *in, T *out,
                       cudaStream_t s) {
    for (int k = 0; k + 3 <= t.L; ++k) {
        const int c = up ? t.L - k : 3 + k;
        tree_translate<T>(ops, nc, cs, cdiv(nc, TR_BM), t, up ? t.m2m_chunk0[c] : t.l2l_chunk0[c],
                          up ? t.m2m_nchunk[c] : t.l2l_nchunk[c], in, out, s);
    }
}

bool use_tc_m2l(const Mesh &m) {
    if (!tc_m2l_available(m)) return false;
    return m.opt.m2l_mode == BEM_M2L_TC || m.opt.m2l_mode == BEM_M2L_AUTO;
}

template <class T>
static void m2l_dense(Mesh &m, const Tree &t, const T *Oop, int nc, int cs, int rblocks, size_t trsm,
                      T *M, T *L, bool timed = false);

// With `apply` set (the collocation K' product), the pass ends in the
// operator's epilogue y = x + Ehat (K'x + table x) instead of writing K'x.
struct ApplyA {
    const double *x;
    double *y;
};

template <class T>
static void run_pass(Mesh &m, const Tree &t, SrcKind sk, TgtKind tk, const double *dens,
                     double *out, bool timed, const ApplyA *apply = nullptr) {
    using B = PassBufs<T>;
    cudaStream_t s = m.stream;
    const TreeView tv = view(t);
    const Tables &tb = tables_for(m, t);
    const int p = m.opt.p;
    const int nc = (p + 1) * (p + 1);
    const int W = 2 * p + 1, W2 = 4 * p + 1;
    const double h = m.side / (double)(1 << t.L);
    const T inv_h = (T)(1.0 / h);
    const int64_t ntgt = (tk == TGT_CEN_DN) ? m.np : (tk == TGT_QUAD_DN ? m.nqp : m.nc);
    const bool far = !(m.opt.flags & BEM_FLAG_NO_FAR) && t.L >= 2;
    const bool near = !(m.opt.flags & BEM_FLAG_NO_NEAR);
    const typename V4T<T>::t *srec = (sk == SRC_QUAD) ? B::qp(m) : B::chg(m);
    const typename V4T<T>::t *trec = (tk == TGT_CEN_DN) ? B::cen(m) : (tk == TGT_QUAD_DN ? B::qp(m) : B::chg(m));
    const typename V4T<T>::t *nrec = (tk == TGT_QUAD_DN) ? B::nrmq(m) : B::nrm(m);
    if (tk == TGT_QUAD_DN && !nrec) throw Error(BEM_EUNSUPPORTED, "quadrature-point normals not built (galerkin = 0)");
    T *far_b = B::far(m), *near_b = B::near(m);
    ev_rec(m, timed, 0);
    const int *qpanel = m.qp_panel.p;
    // The near field (compute bound) runs on a second stream next to the far
    // field's chain of small, latency-bound launches; with phase timing on,
    // everything stays on one stream so each phase is timed alone.
    const bool conc = near && m.stream2 && !(timed && m.tm.on);
    bool near_done = false, joined = false, epi_done = false;
    if (timed) m.tm.near_before_l2p = false;
    // The collocation product's epilogue: the near field carries the FP64
    // near-singular table (out in FP64), L2P (or a last elementwise kernel)
    // writes y = x + Ehat K' x.
    const bool tab_on = apply && m.nt_nnz > 0 && !(m.opt.flags & (BEM_FLAG_NO_NEARTAB | BEM_FLAG_NO_NEAR));
    NearTab ntab{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (apply && near) {
        if (m.near64.n < (size_t)m.np) throw Error(BEM_ECUDA, "near-field FP64 buffer missing");
        ntab = NearTab{tab_on ? m.nt_off.p : nullptr, m.nt_col.p, m.nt_val.p, apply->x, m.near64.p};
    }
    auto launch_near = [&](cudaStream_t ss) {
        const T hh = (T)h;
        // strength records (P2M forms its own strengths)
        typename V4T<T>::t *strec = B::str(m);
        const int64_t ns = (sk == SRC_QUAD) ? m.nqp : m.nc;
        const bool tn = timed && m.tm.on && m.tm.nev[0];
        if (tn) BEM_CUDA(cudaEventRecord(m.tm.nev[0], ss));
        if (ns > 0) {
            if (sk == SRC_QUAD) k_strength_pairs<T, SRC_QUAD><<<t.nleaf, 128, 0, ss>>>(tv, srec, qpanel, dens, strec);
            else k_strength_pairs<T, SRC_CHARGE><<<t.nleaf, 128, 0, ss>>>(tv, srec, nullptr, dens, strec);
            BEM_CHECK_LAUNCH();
        }
        if (tn) BEM_CUDA(cudaEventRecord(m.tm.nev[1], ss));
        // 128-thread CTAs when the average leaf holds at most 32 targets
        const bool small = ntgt <= (int64_t)32 * t.nleaf;
        // (the dynamic tile buffers plus at most 9 KB of static arrays; above
        // 48 KB in all the kernel needs the opt-in)
        const int wk = sk == SRC_QUAD ? 0 : 1;
        if (!t.p2p_hdr[wk].p) throw Error(BEM_ECUDA, "near field: work list missing");
        const P2PList wl{t.p2p_hdr[wk].p, t.p2p_rec[wk].p};
        auto go = [&](auto k128, auto k256) {
            if (small) {
                constexpr size_t sm = p2p_smem<T, 128>();
                if (sm + 9216 > 48 * 1024) ensure_smem_attr(reinterpret_cast<const void *>(k128), sm);
                k128<<<t.nleaf, 128, sm, ss>>>(wl, trec, nrec, strec, hh, near_b, ntab);
            } else {
                constexpr size_t sm = p2p_smem<T, 256>();
                if (sm + 9216 > 48 * 1024) ensure_smem_attr(reinterpret_cast<const void *>(k256), sm);
                k256<<<t.nleaf, 256, sm, ss>>>(wl, trec, nrec, strec, hh, near_b, ntab);
            }
        };
        const bool wide = t.ws == 2;
        if (t.ws != 1 && t.ws != 2) throw Error(BEM_EUNSUPPORTED, "near field: separation not built");
        if (wide && (sk == SRC_QUAD && tk == TGT_CEN_DN || sk == SRC_QUAD && tk == TGT_QUAD_DN))
            throw Error(BEM_EUNSUPPORTED, "the panel tree is separated by one cell");
        if (sk == SRC_QUAD && tk == TGT_CEN_DN)
            go(k_p2p<T, SRC_QUAD, TGT_CEN_DN, 128>, k_p2p<T, SRC_QUAD, TGT_CEN_DN, 256>);
        else if (sk == SRC_QUAD && tk == TGT_QUAD_DN)
            go(k_p2p<T, SRC_QUAD, TGT_QUAD_DN, 128>, k_p2p<T, SRC_QUAD, TGT_QUAD_DN, 256>);
        else if (sk == SRC_CHARGE && tk == TGT_CEN_DN) {
            if (wide) go(k_p2p<T, SRC_CHARGE, TGT_CEN_DN, 128, 125>, k_p2p<T, SRC_CHARGE, TGT_CEN_DN, 256, 125>);
            else go(k_p2p<T, SRC_CHARGE, TGT_CEN_DN, 128>, k_p2p<T, SRC_CHARGE, TGT_CEN_DN, 256>);
        } else if (sk == SRC_QUAD && tk == TGT_CHG_PHI) {
            if (wide) go(k_p2p<T, SRC_QUAD, TGT_CHG_PHI, 128, 125>, k_p2p<T, SRC_QUAD, TGT_CHG_PHI, 256, 125>);
            else go(k_p2p<T, SRC_QUAD, TGT_CHG_PHI, 128>, k_p2p<T, SRC_QUAD, TGT_CHG_PHI, 256>);
        } else if (sk == SRC_CHARGE && tk == TGT_QUAD_DN) {
            if (wide) go(k_p2p<T, SRC_CHARGE, TGT_QUAD_DN, 128, 125>, k_p2p<T, SRC_CHARGE, TGT_QUAD_DN, 256, 125>);
            else go(k_p2p<T, SRC_CHARGE, TGT_QUAD_DN, 128>, k_p2p<T, SRC_CHARGE, TGT_QUAD_DN, 256>);
        } else
            throw Error(BEM_EUNSUPPORTED, "near field: source/target combination not built");
        BEM_CHECK_LAUNCH();
        if (tn) BEM_CUDA(cudaEventRecord(m.tm.nev[2], ss));
    };
    // The near field forks off after the upward sweep (P2M, M2M): the M2L
    // kernel holds every SM by itself (one CTA with ~225 KB of shared memory
    // each) and runs first at the highest priority, and the near field's CTAs
    // fill the SMs around the latency-bound launches before and after it.
    // Measured on the 81,920-panel product: 0.312 ms forked here, 0.319 ms
    // forked before P2M, 0.339 ms after M2L, 0.342 ms one after the other.
    auto fork_near = [&]() {
        BEM_CUDA(cudaEventRecord(m.ev_fork, s));
        BEM_CUDA(cudaStreamWaitEvent(m.stream2, m.ev_fork, 0));
        launch_near(m.stream2);
        BEM_CUDA(cudaEventRecord(m.ev_join, m.stream2));
    };
    if (conc && !far) fork_near();
    if (far) {
        T *M = B::M(m), *L = B::L(m);
        const int cs = cell_stride(p);
        const bool dense = m.opt.m2l_mode != BEM_M2L_DIRECT;
        const int rblocks = cdiv(nc, TR_BM);
        const size_t trsm = translate_smem<T, TR_BN_M2L>();
        if (dense) set_smem<T>(k_translate<T, TR_BN_M2L, TR_THREADS>, trsm);
        // P2M
        p2m_leaves<T>(tv, t.nleaf, sk, srec, qpanel, dens, p, cs, inv_h, M, s);
        ev_rec(m, timed, 1);
        // M2M: parents at levels L-1 .. 2
        if (dense) {
            if (t.L >= 3)
                BEM_CUDA(cudaMemsetAsync(M + (size_t)t.lvl_off[2] * cs, 0,
                                         (size_t)(t.lvl_off[t.L] - t.lvl_off[2]) * cs * sizeof(T), s));
            tree_sweep<T>(m, B::Om2m(tb), nc, cs, t, true, M, M, s);
        } else {
            const size_t sm = 2 * (size_t)(p + 1) * W * sizeof(cpx<T>);
            set_smem<T>(k_m2m<T>, sm);
            for (int l = t.L - 1; l >= 2; --l) {
                const int cnt = t.lvl_off[l + 1] - t.lvl_off[l];
                if (cnt > 0) k_m2m<T><<<cnt, 160, sm, s>>>(tv, t.lvl_off[l], B::R(tb), p, cs, M);
                BEM_CHECK_LAUNCH();
            }
        }
        ev_rec(m, timed, 2);
        if (conc) fork_near();
        // M2L: every cell at levels 2..L
        if (dense) {
            m2l_dense<T>(m, t, B::Om2l(tb), nc, cs, rblocks, trsm, M, L, timed);
        } else {
            const size_t sm = ((size_t)(p + 1) * W + (size_t)(2 * p + 1) * W2) * sizeof(cpx<T>);
            set_smem<T>(k_m2l<T>, sm);
            const int first = t.lvl_off[2];
            const int cnt = t.ncell - first;
            if (cnt > 0) k_m2l<T><<<cnt, 160, sm, s>>>(tv, first, B::I(tb), p, cs, M, L);
            BEM_CHECK_LAUNCH();
        }
        ev_rec(m, timed, 3);
        // L2L: children at levels 3..L
        if (dense) {
            tree_sweep<T>(m, B::Ol2l(tb), nc, cs, t, false, L, L, s);
        } else {
            const size_t sm = 2 * (size_t)(p + 1) * W * sizeof(cpx<T>);
            set_smem<T>(k_l2l<T>, sm);
            for (int l = 3; l <= t.L; ++l) {
                const int cnt = t.lvl_off[l + 1] - t.lvl_off[l];
                if (cnt > 0) k_l2l<T><<<cnt, 160, sm, s>>>(tv, t.lvl_off[l], B::R(tb), p, cs, L);
                BEM_CHECK_LAUNCH();
            }
        }
        ev_rec(m, timed, 4);
        // L2P, carrying the epilogue when the product asks for it; the near
        // field must then be complete (with phase timing on it runs here)
        bool done = false;
        if (apply) {
            if (near && !conc) {
                launch_near(s);
                near_done = true;
                ev_rec(m, timed, 5);
                m.tm.near_before_l2p = true;
            }
            if (near && conc) BEM_CUDA(cudaStreamWaitEvent(s, m.ev_join, 0));
            joined = true;
            const ApplyEpi epi{apply->x, near ? m.near64.p : nullptr, apply->y, m.ehat};
            done = epi_done = l2p_leaves_c<T>(tv, t.nleaf, l2p_threads(ntgt, t.nleaf), tk, p, trec, nrec, cs,
                                              inv_h, L, far_b, s, epi);
        }
        if (!done && !l2p_leaves_c<T>(tv, t.nleaf, l2p_threads(ntgt, t.nleaf), tk, p, trec, nrec, cs, inv_h, L,
                                      far_b, s)) {
            const size_t sm = (size_t)(p + 1) * W * sizeof(cpx<T>);
            if (tk == TGT_CEN_DN) {
                auto kern = k_l2p<T, TGT_CEN_DN>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, l2p_threads(ntgt, t.nleaf), sm, s>>>(tv, trec, nrec, p, cs, inv_h, L, far_b);
            } else if (tk == TGT_QUAD_DN) {
                auto kern = k_l2p<T, TGT_QUAD_DN>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, l2p_threads(ntgt, t.nleaf), sm, s>>>(tv, trec, nrec, p, cs, inv_h, L, far_b);
            } else {
                auto kern = k_l2p<T, TGT_CHG_PHI>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, l2p_threads(ntgt, t.nleaf), sm, s>>>(tv, trec, nrec, p, cs, inv_h, L, far_b);
            }
            BEM_CHECK_LAUNCH();
        }
        ev_rec(m, timed, near_done ? 6 : 5);
    } else {
        for (int k = 1; k <= 5; ++k) ev_rec(m, timed, k);
    }
    if (near && !conc && !near_done) launch_near(s);
    if (!near_done) ev_rec(m, timed, 6);
    if (near && conc && !joined) BEM_CUDA(cudaStreamWaitEvent(s, m.ev_join, 0));
    if (epi_done) {
        // y was written by L2P
    } else if (apply) {
        k_apply_far_near<T><<<cdiv(m.np, 256), 256, 0, s>>>(apply->x, far ? far_b : nullptr, near ? m.near64.p : nullptr,
                                                            m.ehat, m.np, apply->y);
    } else if (tk == TGT_QUAD_DN) {
        // Galerkin rows: the rule's average over each panel of its points' values
        build_qp_of_panel(m);
        k_panel_reduce<T><<<cdiv(m.np, 256), 256, 0, s>>>(far ? far_b : nullptr, near ? near_b : nullptr,
                                                          m.qp_of_panel.p, m.qw64.p, (int)m.nq, m.np, out,
                                                          m.area64.p);
    } else {
        k_combine<T><<<cdiv(ntgt, 256), 256, 0, s>>>(far ? far_b : nullptr, near ? near_b : nullptr,
                                                      ntgt, 1.0 / FOUR_PI, out);
    }
    BEM_CHECK_LAUNCH();
}


void build_qp_of_panel(Mesh &m);

template <class T>
static void near_table_impl(Mesh &m, const double *exact_pan) {
    using B = PassBufs<T>;
    cudaStream_t s = m.stream;
    const Tree &t = m.tp;
    const int64_t np = m.np;
    const int nq = (int)m.nq;
    if (nq != 1 && nq != 7) throw Error(BEM_EUNSUPPORTED, "near-singular table: rule of 1 or 7 points");
    DArray<int> leaf_of, cnt, row;
    StepTimer st(s);
    leaf_of.alloc(np);
    cnt.alloc(np + 1);
    k_leaf_of<<<t.nleaf, 128, 0, s>>>(t.cen_beg.p, t.nleaf, leaf_of.p);
    BEM_CHECK_LAUNCH();
    build_qp_of_panel(m);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (np + 1) * sizeof(int), s));
    k_near_pairs<<<cdiv(np, 128), 128, 0, s>>>(np, t.nbr_off.p, t.nbr.p, t.cen_beg.p, m.cen64.p, m.area64.p,
                                               leaf_of.p, nullptr, cnt.p, nullptr, nullptr);
    BEM_CHECK_LAUNCH();
    m.nt_off.alloc(np + 1);
    exclusive_scan_int(cnt.p, m.nt_off.p, (int)np + 1, s);
    int nnz = 0;
    BEM_CUDA(cudaMemcpyAsync(&nnz, m.nt_off.p + np, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    st.mark("  near-singular table: pairs counted");
    m.nt_nnz = nnz;
    m.nt_col.alloc(nnz);
    m.nt_val.alloc(nnz);
    row.alloc(nnz);
    k_near_pairs<<<cdiv(np, 128), 128, 0, s>>>(np, t.nbr_off.p, t.nbr.p, t.cen_beg.p, m.cen64.p, m.area64.p,
                                               leaf_of.p, m.nt_off.p, nullptr, m.nt_col.p, row.p);
    BEM_CHECK_LAUNCH();
    const int shift = 3 * (MORTON_BITS - t.L);
    const double h = m.side / (double)(1 << t.L);
    if (nnz > 0) {
        auto kern = nq == 7 ? k_near_values<T, 7> : k_near_values<T, 1>;
        kern<<<cdiv(nnz, 128), 128, 0, s>>>((int64_t)nnz, m.nt_col.p, row.p, t.ijk.p, t.leaf0, m.qp_key.p, shift, h,
                                            m.cen64.p, m.nrm64.p, m.qpg64.p, m.qw64.p, m.qp_of_panel.p, B::cen(m),
                                            B::nrm(m), B::qp(m), leaf_of.p, m.nt_val.p, exact_pan, m.cen_perm.p);
        BEM_CHECK_LAUNCH();
    }
    BEM_CUDA(cudaStreamSynchronize(s));  // the temporaries are released on return
    st.mark("  near-singular table: values");
}

// The quadrature points of each sorted panel, in the rule's order, as
// positions in the sorted quadrature array (built with the geometry; see
// build_geometry_and_trees).
void build_qp_of_panel(Mesh &m) {
    if (m.qp_of_panel.n < (size_t)m.nqp || m.nqp == 0)
        throw Error(BEM_ECUDA, "the quadrature points of the panels were not built");
}

// CSR transpose of the near-singular table (for K'^T), on the device:
// column counts, their scan, a fill with one cursor per column, then each
// column's entries put in increasing row order (a few dozen per column), so
// that the transposed product adds them in a fixed order.
__global__ void k_col_count(const int *col, int64_t nnz, int *cnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(cnt + col[e], 1);
}

__global__ void k_col_fill(const int *off, const int *col, const double *val, int64_t np, int *cursor, int *tcol,
                           double *tval) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    for (int e = off[i]; e < off[i + 1]; ++e) {
        const int d = atomicAdd(cursor + col[e], 1);
        tcol[d] = (int)i;
        tval[d] = val[e];
    }
}

__global__ void k_col_sort(const int *toff, int64_t np, int *tcol, double *tval) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int b = toff[j], e = toff[j + 1];
    for (int a = b + 1; a < e; ++a) {  // insertion sort by row
        const int c = tcol[a];
        const double v = tval[a];
        int k = a - 1;
        while (k >= b && tcol[k] > c) {
            tcol[k + 1] = tcol[k];
            tval[k + 1] = tval[k];
            --k;
        }
        tcol[k + 1] = c;
        tval[k + 1] = v;
    }
}

void transpose_near_table(Mesh &m) {
    if (m.ntT_ok) return;
    cudaStream_t s = m.stream;
    const int64_t np = m.np, nnz = m.nt_nnz;
    DArray<int> cnt, cursor;
    cnt.alloc(np + 1);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (np + 1) * sizeof(int), s));
    if (nnz > 0) {
        k_col_count<<<cdiv(nnz, 256), 256, 0, s>>>(m.nt_col.p, nnz, cnt.p);
        BEM_CHECK_LAUNCH();
    }
    m.ntT_off.alloc(np + 1);
    exclusive_scan_int(cnt.p, m.ntT_off.p, (int)np + 1, s);
    m.ntT_col.alloc(nnz);
    m.ntT_val.alloc(nnz);
    if (nnz > 0) {
        cursor.alloc(np + 1);
        BEM_CUDA(cudaMemcpyAsync(cursor.p, m.ntT_off.p, (np + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
        k_col_fill<<<cdiv(np, 256), 256, 0, s>>>(m.nt_off.p, m.nt_col.p, m.nt_val.p, np, cursor.p, m.ntT_col.p,
                                                 m.ntT_val.p);
        BEM_CHECK_LAUNCH();
        k_col_sort<<<cdiv(np, 256), 256, 0, s>>>(m.ntT_off.p, np, m.ntT_col.p, m.ntT_val.p);
        BEM_CHECK_LAUNCH();
    }
    BEM_CUDA(cudaStreamSynchronize(s));  // the counters are released on return
    m.ntT_ok = true;
}

// Per-quadrature-point normals (the normal of the point's panel) in the
// sorted quadrature order: relative records like nrm32 / nrm64r and absolute
// f64 triples.
template <class V>
__global__ void k_qp_normals(const int *qp_panel, int64_t nqp, const V *nrm_rec, const double *nrm64, V *out_rec,
                             double *out64) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nqp) return;
    const int j = qp_panel[k];
    out_rec[k] = nrm_rec[j];
    for (int c = 0; c < 3; ++c) out64[3 * k + c] = nrm64[3 * j + c];
}

void build_galerkin_geometry(Mesh &m) {
    cudaStream_t s = m.stream;
    build_qp_of_panel(m);
    m.nrmq64.alloc((size_t)m.nqp * 3);
    m.gq_tmp.alloc((size_t)m.nqp);
    if (m.opt.precision == BEM_MIXED) {
        m.nrmq32.alloc(m.nqp);
        k_qp_normals<float4><<<cdiv(m.nqp, 256), 256, 0, s>>>(m.qp_panel.p, m.nqp, m.nrm32.p, m.nrm64.p,
                                                             m.nrmq32.p, m.nrmq64.p);
    } else {
        m.nrmq64r.alloc(m.nqp);
        k_qp_normals<double4><<<cdiv(m.nqp, 256), 256, 0, s>>>(m.qp_panel.p, m.nqp, m.nrm64r.p, m.nrm64.p,
                                                              m.nrmq64r.p, m.nrmq64.p);
    }
    BEM_CHECK_LAUNCH();
}

// Near-singular table of the Galerkin rows.  For panel i and each panel j
// whose centroid lies within 2.5 sqrt(A_i) (j != i), the correction
//   D_ij = sum_q w_iq [ exact_j(y_iq) - sum_q' A_j w_q' dn(y_iq; y_jq') ] / (4 pi)
// (w_iq = qw / A_i the rule's weights on panel i, exact_j the exact
// flat-triangle integral of the normal field at y_iq with normal n_i) takes
// the pair from its quadrature value, which the near field and the
// expansions produce, to the exact inner integral.
__global__ void k_near_table_galerkin(int64_t np, int nq, const int *nbr_off, const int *nbr, const int *cen_beg,
                                      const int *leaf_of_cen, const double *cen64, const double *nrm64,
                                      const double *area64, const double *qpg64, const double *qw64,
                                      const int *qp_of_panel, const double *pan, const int *perm,
                                      const int *off, int *cnt, int *col, double *val) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int T_ = leaf_of_cen[i];
    const double ci[3] = {cen64[3 * i], cen64[3 * i + 1], cen64[3 * i + 2]};
    const double ni[3] = {nrm64[3 * i], nrm64[3 * i + 1], nrm64[3 * i + 2]};
    const double tau = 2.5 * sqrt(area64[i]);
    int n = 0;
    const bool fill = off != nullptr;
    const int base = fill ? off[i] : 0;
    for (int e = nbr_off[T_]; e < nbr_off[T_ + 1]; ++e) {
        const int S = nbr[e];
        for (int j = cen_beg[S]; j < cen_beg[S + 1]; ++j) {
            if (j == i) continue;  // outer and inner points in one plane: nothing
            const double dx = ci[0] - cen64[3 * j], dy = ci[1] - cen64[3 * j + 1], dz = ci[2] - cen64[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz > tau * tau) continue;
            if (fill) {
                double acc = 0.0;
                for (int q = 0; q < nq; ++q) {
                    const int k = qp_of_panel[i * nq + q];
                    const double t[3] = {qpg64[3 * k], qpg64[3 * k + 1], qpg64[3 * k + 2]};
                    double quad = 0.0;
                    for (int q2 = 0; q2 < nq; ++q2) {
                        const int k2 = qp_of_panel[(int64_t)j * nq + q2];
                        const double ex = t[0] - qpg64[3 * k2], ey = t[1] - qpg64[3 * k2 + 1],
                                     ez = t[2] - qpg64[3 * k2 + 2];
                        const double r2 = ex * ex + ey * ey + ez * ez;
                        quad += -qw64[k2] * (ex * ni[0] + ey * ni[1] + ez * ni[2]) / (r2 * sqrt(r2));
                    }
                    const double ex = tri_normal_field_4pi(t, ni, pan + 9 * (int64_t)perm[j]);
                    acc += qw64[k] / area64[i] * (ex - quad);
                }
                col[base + n] = j;
                val[base + n] = acc / FOUR_PI;
            }
            ++n;
        }
    }
    if (!fill) cnt[i] = n;
}

static void near_table_galerkin(Mesh &m, const double *panels) {
    cudaStream_t s = m.stream;
    const Tree &t = m.tp;
    const int64_t np = m.np;
    DArray<int> leaf_of, cnt;
    leaf_of.alloc(np);
    cnt.alloc(np + 1);
    k_leaf_of<<<t.nleaf, 128, 0, s>>>(t.cen_beg.p, t.nleaf, leaf_of.p);
    BEM_CHECK_LAUNCH();
    build_qp_of_panel(m);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (np + 1) * sizeof(int), s));
    k_near_table_galerkin<<<cdiv(np, 128), 128, 0, s>>>(np, (int)m.nq, t.nbr_off.p, t.nbr.p, t.cen_beg.p, leaf_of.p,
                                                       m.cen64.p, m.nrm64.p, m.area64.p, m.qpg64.p, m.qw64.p,
                                                       m.qp_of_panel.p, panels, m.cen_perm.p, nullptr, cnt.p,
                                                       nullptr, nullptr);
    BEM_CHECK_LAUNCH();
    m.nt_off.alloc(np + 1);
    exclusive_scan_int(cnt.p, m.nt_off.p, (int)np + 1, s);
    int nnz = 0;
    BEM_CUDA(cudaMemcpyAsync(&nnz, m.nt_off.p + np, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    m.nt_nnz = nnz;
    m.nt_col.alloc(nnz);
    m.nt_val.alloc(nnz);
    k_near_table_galerkin<<<cdiv(np, 128), 128, 0, s>>>(np, (int)m.nq, t.nbr_off.p, t.nbr.p, t.cen_beg.p, leaf_of.p,
                                                       m.cen64.p, m.nrm64.p, m.area64.p, m.qpg64.p, m.qw64.p,
                                                       m.qp_of_panel.p, panels, m.cen_perm.p, m.nt_off.p,
                                                       nullptr, m.nt_col.p, m.nt_val.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));
}

void build_near_table(Mesh &m, const double *panels) {
    if (m.opt.galerkin) {  // the Galerkin rows always take the exact near-singular integrals
        near_table_galerkin(m, panels);
        return;
    }
    const double *exact_pan = m.opt.near_table == BEM_NEAR_EXACT ? panels : nullptr;
    if (m.opt.precision == BEM_MIXED) near_table_impl<float>(m, exact_pan);
    else near_table_impl<double>(m, exact_pan);
    m.ntT_ok = false;  // the transpose is built when the transposed product first needs it
}


template <class T>
static void m2l_dense(Mesh &m, const Tree &t, const T *Oop, int nc, int cs, int rblocks, size_t trsm,
                      T *M, T *L, bool timed) {
    // L at levels >= 2 = the M2L sums (cleared first unless written whole)
    if constexpr (std::is_same<T, float>::value) {
        if (use_tc_m2l(m)) {
            m2l_tc(m, t, M, L, timed);
            return;
        }
    }
    BEM_CUDA(cudaMemsetAsync(L + (size_t)t.lvl_off[2] * cs, 0, (size_t)(t.ncell - t.lvl_off[2]) * cs * sizeof(T),
                             m.stream));
    if (t.m2l_nchunk == 0) return;
    dim3 g(t.m2l_nchunk, rblocks);
    k_translate<T, TR_BN_M2L, TR_THREADS><<<g, TR_THREADS, trsm, m.stream>>>(Oop, nc, cs, t.g_chunk.p + t.m2l_chunk0,
                                                                  t.g_out.p, t.g_in.p, M, L);
    BEM_CHECK_LAUNCH();
}

// Galerkin dipole moments per quadrature point: lam of its panel times the
// rule's weight on that panel, w_q = qw / A
__global__ void k_lam_quad(const double *lam, const int *qp_panel, const double *qw, const double *area, int64_t nqp,
                           double *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nqp) return;
    const int j = qp_panel[i];
    out[i] = lam[j] * (qw[i] / area[j]);
}

void galerkin_moments(Mesh &m, const double *lam) {
    if (m.lamq.n < (size_t)m.nqp) m.lamq.alloc(m.nqp);
    k_lam_quad<<<cdiv(m.nqp, 256), 256, 0, m.stream>>>(lam, m.qp_panel.p, m.qw64.p, m.area64.p, m.nqp, m.lamq.p);
    BEM_CHECK_LAUNCH();
}

template <class T>
static void run_pass_t(Mesh &m, const double *lam, double *out) {
    using B = PassBufs<T>;
    cudaStream_t s = m.stream;
    const Tree &t = m.tp;
    const TreeView tv = view(t);
    const Tables &tb = tables_for(m, t);
    const int p = m.opt.p;
    const int nc = (p + 1) * (p + 1);
    const int cs = cell_stride(p);
    const double h = m.side / (double)(1 << t.L);
    const T inv_h = (T)(1.0 / h);
    const bool far = !(m.opt.flags & BEM_FLAG_NO_FAR) && t.L >= 2;
    const bool near = !(m.opt.flags & BEM_FLAG_NO_NEAR);
    T *far_b = B::far(m), *near_b = B::near(m);
    build_qp_of_panel(m);
    const bool conc = near && m.stream2;
    // the dipoles: lam_i n_i at the collocation points, or for the Galerkin
    // rows lam_i w_q n_i at every quadrature point of panel i
    const int *dbeg = tv.cen_beg;
    const typename V4T<T>::t *drec = B::cen(m), *dnrm = B::nrm(m);
    const double *dlam = lam;
    if (m.opt.galerkin) {
        if (!B::nrmq(m)) throw Error(BEM_ECUDA, "quadrature-point normals not built");
        galerkin_moments(m, lam);
        dbeg = tv.qp_beg;
        drec = B::qp(m);
        dnrm = B::nrmq(m);
        dlam = m.lamq.p;
    }
    auto launch_near = [&](cudaStream_t ss) {
        BEM_CUDA(cudaMemsetAsync(near_b, 0, m.nqp * sizeof(T), ss));
        k_p2p_t<T><<<t.nleaf, P2P_THREADS, 0, ss>>>(tv, dbeg, drec, dnrm, dlam, B::qp(m), (T)h, near_b);
        BEM_CHECK_LAUNCH();
    };
    if (conc) {
        BEM_CUDA(cudaEventRecord(m.ev_fork, s));
        BEM_CUDA(cudaStreamWaitEvent(m.stream2, m.ev_fork, 0));
        launch_near(m.stream2);
        BEM_CUDA(cudaEventRecord(m.ev_join, m.stream2));
    }
    if (far) {
        T *M = B::M(m), *L = B::L(m);
        const int rblocks = cdiv(nc, TR_BM);
        const size_t trsm = translate_smem<T, TR_BN_M2L>();
        set_smem<T>(k_translate<T, TR_BN_M2L, TR_THREADS>, trsm);
        {
            const int th = std::max(32, p2m_threads(p, sizeof(T)));
            const size_t sm = (size_t)th * nc * sizeof(T);
            set_smem<T>(k_p2m_dipole<T>, sm);
            k_p2m_dipole<T><<<t.nleaf, th, sm, s>>>(tv, dbeg, drec, dnrm, dlam, p, cs, inv_h, M);
            BEM_CHECK_LAUNCH();
        }
        if (t.L >= 3)
            BEM_CUDA(cudaMemsetAsync(M + (size_t)t.lvl_off[2] * cs, 0,
                                     (size_t)(t.lvl_off[t.L] - t.lvl_off[2]) * cs * sizeof(T), s));
        tree_sweep<T>(m, B::Om2m(tb), nc, cs, t, true, M, M, s);
        m2l_dense<T>(m, t, B::Om2l(tb), nc, cs, rblocks, trsm, M, L);
        tree_sweep<T>(m, B::Ol2l(tb), nc, cs, t, false, L, L, s);
        if (!l2p_leaves_c<T>(tv, t.nleaf, l2p_threads(m.nqp, t.nleaf), TGT_QUAD_PHI, p, B::qp(m), B::nrm(m), cs,
                             inv_h, L, far_b, s)) {
            const size_t sm = (size_t)(p + 1) * (2 * p + 1) * sizeof(cpx<T>);
            auto kern = k_l2p<T, TGT_QUAD_PHI>;
            set_smem<T>(kern, sm);
            kern<<<t.nleaf, l2p_threads(m.nqp, t.nleaf), sm, s>>>(tv, B::qp(m), B::nrm(m), p, cs, inv_h, L, far_b);
            BEM_CHECK_LAUNCH();
        }
    }
    if (near && !conc) launch_near(s);
    if (near && conc) BEM_CUDA(cudaStreamWaitEvent(s, m.ev_join, 0));
    k_panel_reduce<T><<<cdiv(m.np, 256), 256, 0, s>>>(far ? far_b : nullptr, near ? near_b : nullptr,
                                                      m.qp_of_panel.p, m.qw64.p, (int)m.nq, m.np, out);
    BEM_CHECK_LAUNCH();
}

// Whether a kernel (host stub address, as kernel graph nodes report it) is
// one of the near-field kernels (strength records, P2P) that run on the
// second, low-priority stream.
bool is_near_field_kernel(const void *func) {
    static const void *const near_kernels[] = {
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CEN_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CEN_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_CEN_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_CEN_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CHG_PHI, 128>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CHG_PHI, 256>),

        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CEN_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CEN_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_CEN_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_CEN_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CHG_PHI, 128>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CHG_PHI, 256>),

        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_QUAD_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_QUAD_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_QUAD_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_QUAD_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_QUAD_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_QUAD_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_QUAD_DN, 128>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_QUAD_DN, 256>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_CEN_DN, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_CEN_DN, 256, 125>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CHG_PHI, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_QUAD, TGT_CHG_PHI, 256, 125>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_QUAD_DN, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<float, SRC_CHARGE, TGT_QUAD_DN, 256, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_CEN_DN, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_CEN_DN, 256, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CHG_PHI, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_QUAD, TGT_CHG_PHI, 256, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_QUAD_DN, 128, 125>),
        reinterpret_cast<const void *>(k_p2p<double, SRC_CHARGE, TGT_QUAD_DN, 256, 125>),
        reinterpret_cast<const void *>(k_strength_pairs<float, SRC_QUAD>),
        reinterpret_cast<const void *>(k_strength_pairs<float, SRC_CHARGE>),
        reinterpret_cast<const void *>(k_strength_pairs<double, SRC_QUAD>),
        reinterpret_cast<const void *>(k_strength_pairs<double, SRC_CHARGE>),
        reinterpret_cast<const void *>(k_p2p_t<float>),
        reinterpret_cast<const void *>(k_p2p_t<double>),
    };
    for (const void *k : near_kernels)
        if (k == func) return true;
    return false;
}

void fmm_pass_t(Mesh &m, const double *lam, double *out) {
    if (m.opt.precision == BEM_MIXED) run_pass_t<float>(m, lam, out);
    else run_pass_t<double>(m, lam, out);
}

void kprime_apply(Mesh &m, const double *xs, double *ys) {
    const ApplyA a{xs, ys};
    if (m.opt.precision == BEM_MIXED) run_pass<float>(m, m.tp, SRC_QUAD, TGT_CEN_DN, xs, nullptr, true, &a);
    else run_pass<double>(m, m.tp, SRC_QUAD, TGT_CEN_DN, xs, nullptr, true, &a);
}

void fmm_pass(Mesh &m, const Tree &t, SrcKind sk, TgtKind tk, const double *dens, double *out,
              bool timed) {
    if (m.opt.precision == BEM_MIXED) run_pass<float>(m, t, sk, tk, dens, out, timed);
    else run_pass<double>(m, t, sk, tk, dens, out, timed);
}

}  // namespace bem
