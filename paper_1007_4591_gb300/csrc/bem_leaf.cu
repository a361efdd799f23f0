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
k_p2m_c(TreeView tv, const typename V4T<T>::t *rec, int cs, T inv_h, T *M) {
    constexpr int NC = (P + 1) * (P + 1);
    constexpr int KC = (NC + 31) / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
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
            s = r.w;
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
static void p2m_launch_c(const TreeView &tv, int nleaf, const typename V4T<T>::t *src, int cs, T inv_h,
                         T *M, cudaStream_t s) {
    constexpr int NC = (P + 1) * (P + 1);
    const size_t sm = std::max<size_t>((size_t)P2M_WARPS * 32 * P2M_RS, (size_t)P2M_WARPS * NC) * sizeof(T);
    auto kern = k_p2m_c<T, SRC, P>;
    leaf_smem(kern, sm);
    kern<<<nleaf, P2M_WARPS * 32, sm, s>>>(tv, src, cs, inv_h, M);
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
