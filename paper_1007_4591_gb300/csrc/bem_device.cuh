// Device-side helpers shared by the translation units of the fast multipole
// passes: precision-generic vector records, complex arithmetic, and the
// regular solid harmonics with the expansion order as a template parameter.
#pragma once

#include "bem_internal.cuh"

namespace bem {

template <class T> struct V4T;
template <> struct V4T<float> { using t = float4; };
template <> struct V4T<double> { using t = double4; };

// Strength of source i of a pass: the record's weight times the density
// (A_j w_q dens[panel] for a quadrature point; dens[k], or the charge stored
// in the record when dens is null, for a charge).
// A null dens means the records already hold the strengths.
template <class T, int SRC>
__device__ __forceinline__ T src_strength(T w, int64_t i, const int *qpanel, const double *dens) {
    if (!dens) return w;
    if constexpr (SRC == SRC_QUAD) return w * (T)dens[qpanel[i]];
    else return (T)dens[i];
}

// The operator's epilogue y = x + Ehat (far + near) / (4 pi), fused into
// the last kernel of the collocation K' product (the near field already
// carries the near-singular table's FP64 correction, times 4 pi).
struct ApplyEpi {
    const double *x;       // the product's input (sorted order)
    const double *near64;  // near field + 4 pi table x (null: no near field)
    double *y;             // output; null: no epilogue
    double ehat;
};

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

// Regular solid harmonics R_n^m(x, y, z), 0 <= m <= n <= P, by the Cartesian
// recurrences (Sec. 2.3 expansions)
//   R_0^0 = 1,  R_m^m = -(x + iy)/(2m) R_{m-1}^{m-1},
//   R_n^m = ((2n - 1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n + m)(n - m)),
// unrolled by template recursion so that every (n, m) step is straight-line
// code whose coefficients are compile-time constants (rounded from double).
// emit(n, m, re, im) receives each value, m-major.
template <class T, int P, int Mo, int N, class F>
__device__ __forceinline__ void rs_column(T z, T r2, T are, T aim, T bre, T bim, F &emit) {
    if constexpr (N <= P) {
        constexpr T c2 = (T)(1.0 / ((double)(N + Mo) * (double)(N - Mo)));
        constexpr T k1 = (T)(2 * N - 1);
        const T c1 = k1 * z;
        const T nre = (c1 * bre - r2 * are) * c2, nim = (c1 * bim - r2 * aim) * c2;
        emit(N, Mo, nre, nim);
        rs_column<T, P, Mo, N + 1>(z, r2, bre, bim, nre, nim, emit);
    }
}

template <class T, int P, int Mo, class F>
__device__ __forceinline__ void rs_sectoral(T x, T y, T z, T r2, T dre, T dim, F &emit) {
    if constexpr (Mo <= P) {
        if constexpr (Mo > 0) {
            constexpr T f = -(T)(1.0 / (2.0 * Mo));
            const T nre = f * (x * dre - y * dim), nim = f * (x * dim + y * dre);
            dre = nre;
            dim = nim;
        }
        emit(Mo, Mo, dre, dim);
        if constexpr (Mo + 1 <= P) {
            const T bre = z * dre, bim = z * dim;
            emit(Mo + 1, Mo, bre, bim);
            rs_column<T, P, Mo, Mo + 2>(z, r2, dre, dim, bre, bim, emit);
        }
        rs_sectoral<T, P, Mo + 1>(x, y, z, r2, dre, dim, emit);
    }
}

template <class T, int P, class F>
__device__ __forceinline__ void regular_solid_c(T x, T y, T z, F &&emit) {
    const T r2 = x * x + y * y + z * z;
    rs_sectoral<T, P, 0>(x, y, z, r2, (T)1, (T)0, emit);
}

// P2M of every leaf with the expansion order dispatched to a compile-time
// instance (p in 1..MAXP); one CTA per leaf, queued on `s`:
//   M[leaf]_n^m = sum over the leaf's sources of s_i conj(R_n^m(y_i - z)) / h^n
// with s_i = src_strength(record weight, i, qpanel, dens).
template <class T>
void p2m_leaves(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src, const int *qpanel,
                const double *dens, int p, int cs, T inv_h, T *M, cudaStream_t s);

// L2P of every leaf with a compile-time expansion order (p in {6, 8, 10,
// 12}); one CTA of nth threads per leaf, queued on `s`.  Returns false (and
// launches nothing) for other orders.  With epi.y set (collocation targets)
// it writes the operator's output y instead of the far field.
template <class T>
bool l2p_leaves_c(const TreeView &tv, int nleaf, int nth, TgtKind tk, int p, const typename V4T<T>::t *tgt,
                  const typename V4T<T>::t *nrm, int cs, T inv_h, const T *L, T *out, cudaStream_t s,
                  ApplyEpi epi = ApplyEpi{nullptr, nullptr, nullptr, 0.0});

}  // namespace bem
