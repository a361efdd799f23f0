// P2M (sources -> multipole of their leaf, Sec. 2.3) with the expansion
// order as a template parameter: fixing p at compile time turns the solid
// harmonic recurrence into straight-line code with folded constants; every
// order 1..MAXP is instantiated and picked at run time.
#include <algorithm>

#include "bem_device.cuh"

namespace bem {

template <class KernelT>
static void leaf_smem(KernelT kern, size_t bytes) {
    if (bytes > 48 * 1024) ensure_smem_attr(reinterpret_cast<const void *>(kern), bytes);
}

// ------------------------------------------------------------------- P2M
// A CTA of `warps` warps owns one leaf; each warp takes 32 points at a time,
// writes their strength-weighted harmonics into its own row buffer (odd row
// stride: the column reads below hit 32 different banks) and every lane adds
// up its columns over the 32 rows in registers.  The warps' column sums are
// added in a fixed order at the end.  Lanes without a point write zero rows.
template <class T, int P>
static constexpr int p2m_row_stride() { return ((P + 1) * (P + 1)) | 1; }

template <class T, int SRC, int P>
__global__ void __launch_bounds__(128)
k_p2m_c(TreeView tv, const typename V4T<T>::t *rec, int cs, T inv_h, T *M) {
    constexpr int NC = (P + 1) * (P + 1);
    constexpr int RS = p2m_row_stride<T, P>();
    constexpr int KC = (NC + 31) / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *buf = sm + (size_t)w * 32 * RS;
    T *row = buf + lane * RS;
    const int leaf = blockIdx.x;
    const int *beg = SRC == SRC_QUAD ? tv.qp_beg : tv.chg_beg;
    const int b = beg[leaf], e = beg[leaf + 1];
    T acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = 0;
    for (int base = b + w * 32; base < e; base += nw * 32) {
        const int i = base + lane;
        T x = 0, y = 0, z = 0, s = 0;
        if (i < e) {
            const typename V4T<T>::t r = rec[i];
            x = r.x * inv_h;
            y = r.y * inv_h;
            z = r.z * inv_h;
            s = r.w;
        }
        regular_solid_c<T, P>(x, y, z, [&](int n, int m, T re, T im) {
            if (m == 0) row[n * n] = s * re;
            else {
                row[n * n + 2 * m - 1] = s * re;
                row[n * n + 2 * m] = -s * im;
            }
        });
        __syncwarp();
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int c = lane + 32 * k;
            if (c < NC) {
                T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    s0 += buf[j * RS + c];
                    s1 += buf[(j + 1) * RS + c];
                    s2 += buf[(j + 2) * RS + c];
                    s3 += buf[(j + 3) * RS + c];
                }
                acc[k] += (s0 + s1) + (s2 + s3);
            }
        }
        __syncwarp();
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        if (c < NC) sm[w * NC + c] = acc[k];
    }
    __syncthreads();
    T *out = M + (size_t)(tv.leaf0 + leaf) * cs;
    for (int c = threadIdx.x; c < NC; c += blockDim.x) {
        T a = 0;
        for (int v = 0; v < nw; ++v) a += sm[v * NC + c];
        out[c] = a;
    }
}


// ------------------------------------------------------------------ launch
template <class T, int SRC, int P>
static void p2m_launch_c(const TreeView &tv, int nleaf, const typename V4T<T>::t *src, int cs, T inv_h,
                         T *M, cudaStream_t s) {
    // as many warps per CTA (up to 4) as keep the row buffers within 96 KB
    constexpr size_t row = (size_t)32 * p2m_row_stride<T, P>() * sizeof(T);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (96 * 1024) / row));
    const size_t sm = warps * row;
    auto kern = k_p2m_c<T, SRC, P>;
    leaf_smem(kern, sm);
    kern<<<nleaf, warps * 32, sm, s>>>(tv, src, cs, inv_h, M);
    BEM_CHECK_LAUNCH();
}

template <class T, int P = 1>
static void p2m_dispatch(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src, int p,
                         int cs, T inv_h, T *M, cudaStream_t s) {
    if constexpr (P <= MAXP) {
        if (p != P) return p2m_dispatch<T, P + 1>(tv, nleaf, sk, src, p, cs, inv_h, M, s);
        if (sk == SRC_QUAD) p2m_launch_c<T, SRC_QUAD, P>(tv, nleaf, src, cs, inv_h, M, s);
        else if (sk == SRC_CHARGE) p2m_launch_c<T, SRC_CHARGE, P>(tv, nleaf, src, cs, inv_h, M, s);
        else throw Error(BEM_EUNSUPPORTED, "P2M source kind not built");
    } else {
        throw Error(BEM_EINVAL, "expansion order out of range");
    }
}

template <class T>
void p2m_leaves(const TreeView &tv, int nleaf, SrcKind sk, const typename V4T<T>::t *src, int p, int cs,
                T inv_h, T *M, cudaStream_t s) {
    if (nleaf > 0) p2m_dispatch<T>(tv, nleaf, sk, src, p, cs, inv_h, M, s);
}

template void p2m_leaves<float>(const TreeView &, int, SrcKind, const float4 *, int, int, float, float *,
                                cudaStream_t);
template void p2m_leaves<double>(const TreeView &, int, SrcKind, const double4 *, int, int, double, double *,
                                 cudaStream_t);
}  // namespace bem
