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
#include <cmath>
#include <cstring>

#include "bem_internal.cuh"

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

template <class T> struct V4T;
template <> struct V4T<float> { using t = float4; };
template <> struct V4T<double> { using t = double4; };

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class T>
struct cpx {
    T x, y;
};

template <class T>
__device__ __forceinline__ void cmac(cpx<T> &acc, cpx<T> a, cpx<T> b) {  // acc += a*b
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <class T>
__device__ __forceinline__ void cmac_conjb(cpx<T> &acc, cpx<T> a, cpx<T> b) {  // acc += a*conj(b)
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
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
template <class T, int SRC>
__global__ void k_p2m(TreeView tv, const typename V4T<T>::t *rec, const int *qpanel,
                      const double *dens, int p, T inv_h, T *M) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sh = reinterpret_cast<T *>(smraw);
    const int leaf = blockIdx.x;
    const int *beg = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int b = beg[leaf], e = beg[leaf + 1];
    const int nc = (p + 1) * (p + 1);
    constexpr int MAXACC = 10;  // ceil((MAXP+1)^2 / 32)
    T acc[MAXACC];
#pragma unroll
    for (int k = 0; k < MAXACC; ++k) acc[k] = 0;
    for (int base = b; base < e; base += blockDim.x) {
        const int i = base + threadIdx.x;
        T *row = sh + threadIdx.x * nc;
        if (i < e) {
            const typename V4T<T>::t r = rec[i];
            T s;
            if (SRC == SRC_QUAD) s = r.w * (T)dens[qpanel[i]];
            else s = dens ? (T)dens[i] : r.w;
            regular_solid<T>(r.x * inv_h, r.y * inv_h, r.z * inv_h, p,
                             [&](int n, int m, T re, T im) {
                                 if (m == 0) row[n * n] = s * re;
                                 else {
                                     row[n * n + 2 * m - 1] = s * re;
                                     row[n * n + 2 * m] = -s * im;
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
    T *out = M + (size_t)(tv.leaf0 + leaf) * nc;
    int k = 0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x, ++k) {
#pragma unroll
        for (int q = 0; q < MAXACC; ++q)
            if (q == k) out[c] = acc[q];
    }
}

// ------------------------------------------------------------------- M2M
// Parents [first, last) gather their children's multipoles.
template <class T>
__global__ void k_m2m(TreeView tv, int first, const cpx<T> *Rtab, int p, T *M) {
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
        load_full<T>(M + (size_t)c * nc, p, Mc);
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
        T *out = M + (size_t)cell * nc;
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
__global__ void k_m2l(TreeView tv, int first, const cpx<T> *Itab, int p, const T *M, T *L) {
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
        load_full<T>(M + (size_t)tv.m2l_src[e] * nc, p, Ms);
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
        T *out = L + (size_t)cell * nc;
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
__global__ void k_l2l(TreeView tv, int first, const cpx<T> *Rtab, int p, T *L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1;
    cpx<T> *Lp = reinterpret_cast<cpx<T> *>(smraw);
    cpx<T> *Rd = Lp + (p + 1) * W;
    const int cell = first + blockIdx.x;
    const int nc = (p + 1) * (p + 1);
    const int ntri = (p + 1) * (p + 2) / 2;
    const int t = threadIdx.x;
    const int P = tv.parent[cell];
    load_full<T>(L + (size_t)P * nc, p, Lp);
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
        T *out = L + (size_t)cell * nc;
        if (l == 0) out[k * k] += s * acc.x;
        else {
            out[k * k + 2 * l - 1] += s * acc.x;
            out[k * k + 2 * l] += s * acc.y;
        }
    }
}

// ------------------------------------------------------------------- L2P
template <class T, int TGT>
__global__ void k_l2p(TreeView tv, const typename V4T<T>::t *tgt, const typename V4T<T>::t *nrm,
                      int p, T inv_h, const T *L, T *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = 2 * p + 1;
    cpx<T> *Lf = reinterpret_cast<cpx<T> *>(smraw);
    const int leaf = blockIdx.x;
    const int *beg = TGT == TGT_CEN_DN ? tv.cen_beg : tv.chg_beg;
    const int b = beg[leaf], e = beg[leaf + 1];
    if (b == e) return;
    load_full<T>(L + (size_t)(tv.leaf0 + leaf) * (p + 1) * (p + 1), p, Lf);
    __syncthreads();
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const typename V4T<T>::t r = tgt[i];
        const T x = r.x * inv_h, y = r.y * inv_h, z = r.z * inv_h;
        if (TGT == TGT_CEN_DN) {
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
    const T ri = rsq(r2);
    nd = fma(nx, dx, fma(ny, dy, nz * dz));
    ri3 = ri * ri * ri;
}

template <class T, int SRC, int TGT>
__global__ void __launch_bounds__(P2P_THREADS)
k_p2p(TreeView tv, const typename V4T<T>::t *tgt, const typename V4T<T>::t *nrm,
      const typename V4T<T>::t *src, const int *qpanel, const double *dens, T h, T *out) {
    using V4 = typename V4T<T>::t;
    __shared__ V4 sh[P2P_THREADS];
    __shared__ int s_beg[28], s_cum[28];
    __shared__ T s_off[27][3];
    const int leaf = blockIdx.x;
    const int *tb_ = TGT == TGT_CEN_DN ? tv.cen_beg : tv.chg_beg;
    const int *sb_ = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int tb = tb_[leaf], te = tb_[leaf + 1];
    if (tb == te) return;
    const int nb0 = tv.nbr_off[leaf], nn = tv.nbr_off[leaf + 1] - nb0;
    const int4 ct = tv.ijk[tv.leaf0 + leaf];
    if (threadIdx.x < nn) {
        const int S = tv.nbr[nb0 + threadIdx.x];
        const int4 cs = tv.ijk[tv.leaf0 + S];
        s_beg[threadIdx.x] = sb_[S];
        s_cum[threadIdx.x + 1] = sb_[S + 1] - sb_[S];
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
    int G = 1;
    while (G < 8 && ntgt * G * 2 <= P2P_THREADS) G *= 2;
    const int per = P2P_THREADS / G;
    const int g = threadIdx.x & (G - 1);
    const T EPS = P2PEps<T>::v;
    for (int t0 = 0; t0 < ntgt; t0 += per) {
        const int ti = t0 + threadIdx.x / G;
        const bool valid = ti < ntgt;
        T cx = 0, cy = 0, cz = 0, nx = 0, ny = 0, nz = 0;
        if (valid) {
            const V4 c = tgt[tb + ti];
            cx = c.x;
            cy = c.y;
            cz = c.z;
            if (TGT == TGT_CEN_DN) {
                const V4 nv = nrm[tb + ti];
                nx = nv.x;
                ny = nv.y;
                nz = nv.z;
            }
        }
        T outer = 0;  // sum of per-tile sums (short FP32 accumulations)
        for (int vb = 0; vb < total; vb += P2P_THREADS) {
            __syncthreads();
            const int v = vb + threadIdx.x;
            if (v < total) {
                int lo = 0, hi = nn;  // segment k with s_cum[k] <= v < s_cum[k+1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_cum[mid] <= v) lo = mid;
                    else hi = mid;
                }
                const int si = s_beg[lo] + (v - s_cum[lo]);
                V4 r = src[si];
                T s;
                if (SRC == SRC_QUAD) s = r.w * (T)dens[qpanel[si]];
                else s = dens ? (T)dens[si] : r.w;
                r.x += s_off[lo][0];
                r.y += s_off[lo][1];
                r.z += s_off[lo][2];
                r.w = s;
                sh[threadIdx.x] = r;
            }
            __syncthreads();
            const int cnt = min(P2P_THREADS, total - vb);
            T acc = 0;
            if (valid) {
#pragma unroll 4
                for (int j = g; j < cnt; j += G) {
                    const V4 y = sh[j];
                    const T dx = cx - y.x, dy = cy - y.y, dz = cz - y.z;
                    if (TGT == TGT_CEN_DN) {
                        T nd, ri3;
                        dn_pair<T>(dx, dy, dz, nx, ny, nz, nd, ri3);
                        acc = fma(y.w * nd, ri3, acc);
                    } else {
                        const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, EPS)));
                        acc = fma(y.w, rsq(r2), acc);
                    }
                }
            }
            outer += acc;
        }
        for (int o = G >> 1; o > 0; o >>= 1) outer += __shfl_xor_sync(0xffffffffu, outer, o);
        if (valid && g == 0) out[tb + ti] = (TGT == TGT_CEN_DN) ? -outer : outer;
    }
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
template <class T, bool FILL>
__global__ void k_near_table(int64_t np, int nq, const int *nbr_off, const int *nbr,
                             const int *cen_beg, const int4 *ijk, int leaf0, const uint64_t *cen_key,
                             const uint64_t *qp_key, int shift, double h, const double *cen64,
                             const double *nrm64, const double *area64, const double *qpg64,
                             const double *qw64, const int *qp_of_panel,
                             const typename V4T<T>::t *trec, const typename V4T<T>::t *nrec,
                             const typename V4T<T>::t *srec, const int *leaf_of_cen,
                             const int *off, int *cnt, int *col, double *val) {
    using V4 = typename V4T<T>::t;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int T_ = leaf_of_cen[i];
    const int4 ct = ijk[leaf0 + T_];
    const double ci[3] = {cen64[3 * i], cen64[3 * i + 1], cen64[3 * i + 2]};
    const double ni[3] = {nrm64[3 * i], nrm64[3 * i + 1], nrm64[3 * i + 2]};
    const double tau = 2.5 * sqrt(area64[i]);
    const V4 tr = trec[i], nr = nrec[i];
    int n = 0;
    const int base = FILL ? off[i] : 0;
    for (int e = nbr_off[T_]; e < nbr_off[T_ + 1]; ++e) {
        const int S = nbr[e];
        for (int j = cen_beg[S]; j < cen_beg[S + 1]; ++j) {
            const double dx = ci[0] - cen64[3 * j], dy = ci[1] - cen64[3 * j + 1],
                         dz = ci[2] - cen64[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz > tau * tau) continue;
            if (FILL) {
                double exact = 0.0, rep = 0.0;
                for (int q = 0; q < nq; ++q) {
                    const int k = qp_of_panel[(int64_t)j * nq + q];
                    int a, b, c;
                    {
                        uint64_t key = qp_key[k] >> shift;
                        // decode leaf coordinates of the source point
                        uint64_t x = key;
                        auto cb = [](uint64_t v) {
                            v &= 0x1249249249249249ull;
                            v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
                            v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
                            v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
                            v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
                            v = (v ^ (v >> 32)) & 0x1fffffull;
                            return (int)v;
                        };
                        a = cb(x);
                        b = cb(x >> 1);
                        c = cb(x >> 2);
                    }
                    if (abs(a - ct.x) > 1 || abs(b - ct.y) > 1 || abs(c - ct.z) > 1) continue;
                    if (j != i) {
                        const double ex = ci[0] - qpg64[3 * k], ey = ci[1] - qpg64[3 * k + 1],
                                     ez = ci[2] - qpg64[3 * k + 2];
                        const double r2 = ex * ex + ey * ey + ez * ez;
                        const double r = sqrt(r2);
                        exact += -qw64[k] * (ex * ni[0] + ey * ni[1] + ez * ni[2]) / (r2 * r);
                    }
                    // replay of the near-field kernel for this point
                    V4 y = srec[k];
                    const double hT = (double)(T)h;  // the P2P kernel receives h in T
                    y.x += (T)((double)(a - ct.x) * hT);
                    y.y += (T)((double)(b - ct.y) * hT);
                    y.z += (T)((double)(c - ct.z) * hT);
                    T nd, ri3;
                    dn_pair<T>(tr.x - y.x, tr.y - y.y, tr.z - y.z, nr.x, nr.y, nr.z, nd, ri3);
                    rep += -(double)y.w * (double)nd * (double)ri3;
                }
                col[base + n] = j;
                val[base + n] = (exact - rep) / FOUR_PI;
            }
            ++n;
        }
    }
    if (!FILL) cnt[i] = n;
}

__global__ void k_leaf_of(const int *beg, int nleaf, int *leaf_of) {
    const int l = blockIdx.x;
    for (int i = beg[l] + threadIdx.x; i < beg[l + 1]; i += blockDim.x) leaf_of[i] = l;
}

__global__ void k_qp_of_panel(const int *qp_panel, const uint64_t *dummy, int64_t nqp, int nq,
                              int *slot_cnt, int *qp_of_panel) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nqp) return;
    const int j = qp_panel[k];
    const int s = atomicAdd(&slot_cnt[j], 1);
    qp_of_panel[(int64_t)j * nq + s] = (int)k;
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

static void upload_constants(int dev) {
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

void build_tables(Mesh &m) {
    upload_constants(m.device);
    const int p = m.opt.p;
    const int W = 2 * p + 1, W2 = 4 * p + 1;
    m.tab.p = p;
    // parent/child offsets: child centre minus parent centre over the parent size
    std::vector<double> r8((size_t)8 * (p + 1) * W * 2), tmp;
    for (int o = 0; o < 8; ++o) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = ((o >> k) & 1) ? 0.25 : -0.25;
        host_regular_full(d[0], d[1], d[2], p, tmp);
        std::memcpy(&r8[(size_t)o * (p + 1) * W * 2], tmp.data(), tmp.size() * sizeof(double));
    }
    // M2L offsets: target centre minus source centre over the cell size = -(dx,dy,dz)
    const size_t itot = (size_t)(2 * p + 1) * W2 * 2;
    std::vector<double> it((size_t)NOFFSET * itot, 0.0);
    for (int o = 0; o < NOFFSET; ++o) {
        int dx = o / 49 - 3, dy = (o / 7) % 7 - 3, dz = o % 7 - 3;
        if (std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1) continue;
        host_irregular_full(-dx, -dy, -dz, 2 * p, tmp);
        std::memcpy(&it[(size_t)o * itot], tmp.data(), tmp.size() * sizeof(double));
    }
    if (m.opt.precision == BEM_MIXED) {
        std::vector<float> a(r8.begin(), r8.end()), b(it.begin(), it.end());
        m.tab.Rm2m_f.alloc(a.size());
        m.tab.If_f.alloc(b.size());
        BEM_CUDA(cudaMemcpy(m.tab.Rm2m_f.p, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice));
        BEM_CUDA(cudaMemcpy(m.tab.If_f.p, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        m.tab.Rm2m_d.alloc(r8.size());
        m.tab.If_d.alloc(it.size());
        BEM_CUDA(cudaMemcpy(m.tab.Rm2m_d.p, r8.data(), r8.size() * sizeof(double), cudaMemcpyHostToDevice));
        BEM_CUDA(cudaMemcpy(m.tab.If_d.p, it.data(), it.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
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
    static const cpx<float> *R(Mesh &m) { return reinterpret_cast<const cpx<float> *>(m.tab.Rm2m_f.p); }
    static const cpx<float> *I(Mesh &m) { return reinterpret_cast<const cpx<float> *>(m.tab.If_f.p); }
    static const float4 *cen(Mesh &m) { return m.cen32.p; }
    static const float4 *nrm(Mesh &m) { return m.nrm32.p; }
    static const float4 *qp(Mesh &m) { return m.qp32.p; }
    static const float4 *chg(Mesh &m) { return m.chg32.p; }
};
template <>
struct PassBufs<double> {
    static double *M(Mesh &m) { return m.Md.p; }
    static double *L(Mesh &m) { return m.Ld.p; }
    static double *far(Mesh &m) { return m.far_d.p; }
    static double *near(Mesh &m) { return m.near_d.p; }
    static const cpx<double> *R(Mesh &m) { return reinterpret_cast<const cpx<double> *>(m.tab.Rm2m_d.p); }
    static const cpx<double> *I(Mesh &m) { return reinterpret_cast<const cpx<double> *>(m.tab.If_d.p); }
    static const double4 *cen(Mesh &m) { return m.cen64r.p; }
    static const double4 *nrm(Mesh &m) { return m.nrm64r.p; }
    static const double4 *qp(Mesh &m) { return m.qp64r.p; }
    static const double4 *chg(Mesh &m) { return m.chg64r.p; }
};

static int p2m_threads(int p, size_t elt) {
    const size_t nc = (size_t)(p + 1) * (p + 1);
    int t = 128;
    while (t > 32 && (size_t)t * nc * elt > 96 * 1024) t >>= 1;
    return t;
}

template <class T, class KernelT>
static void set_smem(KernelT kern, size_t bytes) {
    if (bytes > 48 * 1024)
        BEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static void ev_rec(Mesh &m, bool timed, int k) {
    if (timed && m.tm.on) BEM_CUDA(cudaEventRecord(m.tm.ev[k], m.stream));
}

template <class T>
static void run_pass(Mesh &m, const Tree &t, SrcKind sk, TgtKind tk, const double *dens,
                     double *out, bool timed) {
    using B = PassBufs<T>;
    cudaStream_t s = m.stream;
    const TreeView tv = view(t);
    const int p = m.opt.p;
    const int nc = (p + 1) * (p + 1);
    const int W = 2 * p + 1, W2 = 4 * p + 1;
    const double h = m.side / (double)(1 << t.L);
    const T inv_h = (T)(1.0 / h);
    const int64_t ntgt = (tk == TGT_CEN_DN) ? m.np : m.nc;
    const bool far = !(m.opt.flags & BEM_FLAG_NO_FAR) && t.L >= 2;
    const bool near = !(m.opt.flags & BEM_FLAG_NO_NEAR);
    const typename V4T<T>::t *srec = (sk == SRC_QUAD) ? B::qp(m) : B::chg(m);
    const typename V4T<T>::t *trec = (tk == TGT_CEN_DN) ? B::cen(m) : B::chg(m);
    const typename V4T<T>::t *nrec = B::nrm(m);
    T *far_b = B::far(m), *near_b = B::near(m);
    ev_rec(m, timed, 0);
    if (far) {
        T *M = B::M(m), *L = B::L(m);
        // P2M
        {
            const int th = p2m_threads(p, sizeof(T));
            const size_t sm = (size_t)th * nc * sizeof(T);
            if (sk == SRC_QUAD) {
                auto kern = k_p2m<T, SRC_QUAD>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, th, sm, s>>>(tv, srec, m.qp_panel.p, dens, p, inv_h, M);
            } else {
                auto kern = k_p2m<T, SRC_CHARGE>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, th, sm, s>>>(tv, srec, nullptr, dens, p, inv_h, M);
            }
            BEM_CHECK_LAUNCH();
        }
        ev_rec(m, timed, 1);
        // M2M: parents at levels L-1 .. 2
        {
            const size_t sm = 2 * (size_t)(p + 1) * W * sizeof(cpx<T>);
            set_smem<T>(k_m2m<T>, sm);
            for (int l = t.L - 1; l >= 2; --l) {
                const int cnt = t.lvl_off[l + 1] - t.lvl_off[l];
                if (cnt > 0) k_m2m<T><<<cnt, 160, sm, s>>>(tv, t.lvl_off[l], B::R(m), p, M);
                BEM_CHECK_LAUNCH();
            }
        }
        ev_rec(m, timed, 2);
        // M2L: every cell at levels 2..L
        {
            const size_t sm = ((size_t)(p + 1) * W + (size_t)(2 * p + 1) * W2) * sizeof(cpx<T>);
            set_smem<T>(k_m2l<T>, sm);
            const int first = t.lvl_off[2];
            const int cnt = t.ncell - first;
            if (cnt > 0) k_m2l<T><<<cnt, 160, sm, s>>>(tv, first, B::I(m), p, M, L);
            BEM_CHECK_LAUNCH();
        }
        ev_rec(m, timed, 3);
        // L2L: children at levels 3..L
        {
            const size_t sm = 2 * (size_t)(p + 1) * W * sizeof(cpx<T>);
            set_smem<T>(k_l2l<T>, sm);
            for (int l = 3; l <= t.L; ++l) {
                const int cnt = t.lvl_off[l + 1] - t.lvl_off[l];
                if (cnt > 0) k_l2l<T><<<cnt, 160, sm, s>>>(tv, t.lvl_off[l], B::R(m), p, L);
                BEM_CHECK_LAUNCH();
            }
        }
        ev_rec(m, timed, 4);
        // L2P
        {
            const size_t sm = (size_t)(p + 1) * W * sizeof(cpx<T>);
            if (tk == TGT_CEN_DN) {
                auto kern = k_l2p<T, TGT_CEN_DN>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, 128, sm, s>>>(tv, trec, nrec, p, inv_h, L, far_b);
            } else {
                auto kern = k_l2p<T, TGT_CHG_PHI>;
                set_smem<T>(kern, sm);
                kern<<<t.nleaf, 128, sm, s>>>(tv, trec, nrec, p, inv_h, L, far_b);
            }
            BEM_CHECK_LAUNCH();
        }
        ev_rec(m, timed, 5);
    } else {
        for (int k = 1; k <= 5; ++k) ev_rec(m, timed, k);
    }
    if (near) {
        const T hh = (T)h;
        if (sk == SRC_QUAD && tk == TGT_CEN_DN)
            k_p2p<T, SRC_QUAD, TGT_CEN_DN><<<t.nleaf, P2P_THREADS, 0, s>>>(tv, trec, nrec, srec, m.qp_panel.p, dens, hh, near_b);
        else if (sk == SRC_CHARGE && tk == TGT_CEN_DN)
            k_p2p<T, SRC_CHARGE, TGT_CEN_DN><<<t.nleaf, P2P_THREADS, 0, s>>>(tv, trec, nrec, srec, nullptr, dens, hh, near_b);
        else if (sk == SRC_QUAD && tk == TGT_CHG_PHI)
            k_p2p<T, SRC_QUAD, TGT_CHG_PHI><<<t.nleaf, P2P_THREADS, 0, s>>>(tv, trec, nrec, srec, m.qp_panel.p, dens, hh, near_b);
        else
            k_p2p<T, SRC_CHARGE, TGT_CHG_PHI><<<t.nleaf, P2P_THREADS, 0, s>>>(tv, trec, nrec, srec, nullptr, dens, hh, near_b);
        BEM_CHECK_LAUNCH();
    }
    ev_rec(m, timed, 6);
    k_combine<T><<<cdiv(ntgt, 256), 256, 0, s>>>(far ? far_b : nullptr, near ? near_b : nullptr,
                                                  ntgt, 1.0 / FOUR_PI, out);
    BEM_CHECK_LAUNCH();
}


template <class T>
static void near_table_impl(Mesh &m) {
    using B = PassBufs<T>;
    cudaStream_t s = m.stream;
    const Tree &t = m.tp;
    const int64_t np = m.np;
    const int nq = (int)m.nq;
    DArray<int> leaf_of, slot, qop, cnt;
    leaf_of.alloc(np);
    slot.alloc(np);
    qop.alloc(m.nqp);
    cnt.alloc(np + 1);
    k_leaf_of<<<t.nleaf, 128, 0, s>>>(t.cen_beg.p, t.nleaf, leaf_of.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaMemsetAsync(slot.p, 0, np * sizeof(int), s));
    k_qp_of_panel<<<cdiv(m.nqp, 256), 256, 0, s>>>(m.qp_panel.p, nullptr, m.nqp, nq, slot.p, qop.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (np + 1) * sizeof(int), s));
    const int shift = 3 * (MORTON_BITS - t.L);
    const double h = m.side / (double)(1 << t.L);
    k_near_table<T, false><<<cdiv(np, 128), 128, 0, s>>>(
        np, nq, t.nbr_off.p, t.nbr.p, t.cen_beg.p, t.ijk.p, t.leaf0, m.cen_key.p, m.qp_key.p, shift, h,
        m.cen64.p, m.nrm64.p, m.area64.p, m.qpg64.p, m.qw64.p, qop.p, B::cen(m), B::nrm(m), B::qp(m),
        leaf_of.p, nullptr, cnt.p, nullptr, nullptr);
    BEM_CHECK_LAUNCH();
    m.nt_off.alloc(np + 1);
    exclusive_scan_int(cnt.p, m.nt_off.p, (int)np + 1, s);
    int nnz = 0;
    BEM_CUDA(cudaMemcpyAsync(&nnz, m.nt_off.p + np, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    m.nt_nnz = nnz;
    m.nt_col.alloc(nnz);
    m.nt_val.alloc(nnz);
    k_near_table<T, true><<<cdiv(np, 128), 128, 0, s>>>(
        np, nq, t.nbr_off.p, t.nbr.p, t.cen_beg.p, t.ijk.p, t.leaf0, m.cen_key.p, m.qp_key.p, shift, h,
        m.cen64.p, m.nrm64.p, m.area64.p, m.qpg64.p, m.qw64.p, qop.p, B::cen(m), B::nrm(m), B::qp(m),
        leaf_of.p, m.nt_off.p, nullptr, m.nt_col.p, m.nt_val.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));
}

void build_near_table(Mesh &m) {
    if (m.opt.precision == BEM_MIXED) near_table_impl<float>(m);
    else near_table_impl<double>(m);
}

void fmm_pass(Mesh &m, const Tree &t, SrcKind sk, TgtKind tk, const double *dens, double *out,
              bool timed) {
    if (m.opt.precision == BEM_MIXED) run_pass<float>(m, t, sk, tk, dens, out, timed);
    else run_pass<double>(m, t, sk, tk, dens, out, timed);
}

}  // namespace bem
