// Sorting and scans of the tree build (Sec. 3.1: the points are ordered by
// their Morton keys, the tree's cells and lists laid out by prefix sums).
//
// Stable least-significant-digit radix sort, 8-bit digits.  Each pass:
//   1. every block (a tile of RS_TILE keys) counts its digits;
//   2. the counts, laid out [digit][block], are scanned, giving each block
//      the first output position of each digit;
//   3. every block writes its keys in tile order: a warp's lanes with equal
//      digits find each other (match.any) and take consecutive positions after
//      the lower warps' counts of that digit, round after round.
// Keys or positions are not compared across blocks, so the order of equal
// digits is the input order: the sort is stable, and with values it carries
// each key's value along.
//
// Scans are the usual three steps: a block scan of tiles that also writes
// each tile's total, a (recursive) scan of the totals, and the totals added
// back.
#include <cstdint>

#include "bem_internal.cuh"

namespace bem {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K *__restrict__ keys, int64_t n, int shift, int nblk,
                                                        int *__restrict__ hist) {
    __shared__ int h[RS_BINS];
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int64_t i = base + it * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & (RS_BINS - 1))], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) hist[(int64_t)d * nblk + blockIdx.x] = h[d];
}

template <class K, bool VALS>
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const K *__restrict__ kin, const int *__restrict__ vin, K *__restrict__ kout, int *__restrict__ vout,
             int64_t n, int shift, int nblk, const int *__restrict__ off) {
    __shared__ int s_base[RS_BINS];            // next output position of each digit
    __shared__ int s_wcnt[RS_WARPS][RS_BINS];  // this round's count of each digit per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
        s_base[d] = off[(int64_t)d * nblk + blockIdx.x];
        for (int w = 0; w < RS_WARPS; ++w) s_wcnt[w][d] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int64_t i = base + it * RS_THREADS + threadIdx.x;
        const bool ok = i < n;
        const K k = ok ? kin[i] : (K)0;
        int v = 0;
        if (VALS && ok) v = vin[i];
        const int d = ok ? (int)((k >> shift) & (RS_BINS - 1)) : -1;  // lanes past the end group apart
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const bool leader = rank == 0;
        if (ok && leader) s_wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            int pos = s_base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += s_wcnt[w][d];
            kout[pos] = k;
            if (VALS) vout[pos] = v;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < RS_BINS; dd += RS_THREADS) {
            int t = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) t += s_wcnt[w][dd];
            s_base[dd] += t;
        }
        __syncthreads();
        if (ok && leader) s_wcnt[warp][d] = 0;  // cleared by its writer before the next round
        __syncwarp();
    }
}

// ------------------------------------------------------------------ scans
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

// Scan of one tile (each thread owns SC_ITEMS consecutive values); the
// tile's total goes to sums[blockIdx.x] when sums is set.
__global__ void __launch_bounds__(SC_THREADS)
k_scan_tile(const int *__restrict__ in, int *__restrict__ out, int64_t n, int *__restrict__ sums, int inclusive) {
    __shared__ int s_warp[SC_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        tsum += v[k];
    }
    // exclusive scan of the threads' sums: within warps by shuffles, then across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < SC_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SC_THREADS / 32) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    int run = x - tsum + (warp > 0 ? s_warp[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const int e = run;
        run += v[k];
        if (base + k < n) out[base + k] = inclusive ? run : e;
    }
    if (sums && threadIdx.x == SC_THREADS - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int *__restrict__ out, int64_t n, const int *__restrict__ offs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / SC_TILE];
}

static void scan_i32(const int *in, int *out, int64_t n, bool inclusive, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 1) {
        k_scan_tile<<<1, SC_THREADS, 0, s>>>(in, out, n, nullptr, inclusive ? 1 : 0);
        BEM_CHECK_LAUNCH();
        return;
    }
    DArray<int> sums, offs;
    sums.alloc(nb);
    offs.alloc(nb);
    k_scan_tile<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, n, sums.p, inclusive ? 1 : 0);
    BEM_CHECK_LAUNCH();
    scan_i32(sums.p, offs.p, nb, false, s);
    k_scan_add<<<cdiv(n, 256), 256, 0, s>>>(out, n, offs.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));  // the tile totals are released on return
}

void scan_exclusive_i32(const int *in, int *out, int64_t n, cudaStream_t s) { scan_i32(in, out, n, false, s); }
void scan_inclusive_i32(const int *in, int *out, int64_t n, cudaStream_t s) { scan_i32(in, out, n, true, s); }

// ------------------------------------------------------------ radix sort
template <class K>
static void radix_sort(const K *k_in, const int *v_in, K *k_out, int *v_out, int64_t n, int bits, cudaStream_t s) {
    if (n <= 0) return;
    const bool vals = v_in != nullptr;
    const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    const int passes = (bits + 7) / 8;
    DArray<K> kb;
    DArray<int> vb, hist, off;
    kb.alloc(n);
    if (vals) vb.alloc(n);
    hist.alloc((size_t)RS_BINS * nblk);
    off.alloc((size_t)RS_BINS * nblk);
    // ping-pong so that the last pass writes k_out / v_out
    const K *ks = k_in;
    const int *vs = v_in;
    for (int pass = 0; pass < passes; ++pass) {
        const bool last = pass == passes - 1;
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        K *kd = to_out ? k_out : kb.p;
        int *vd = vals ? (to_out ? v_out : vb.p) : nullptr;
        if (!last && ks == kd) throw Error(BEM_ECUDA, "radix sort: in-place pass");
        k_rs_hist<K><<<nblk, RS_THREADS, 0, s>>>(ks, n, 8 * pass, nblk, hist.p);
        BEM_CHECK_LAUNCH();
        scan_exclusive_i32(hist.p, off.p, (int64_t)RS_BINS * nblk, s);
        if (vals) k_rs_scatter<K, true><<<nblk, RS_THREADS, 0, s>>>(ks, vs, kd, vd, n, 8 * pass, nblk, off.p);
        else k_rs_scatter<K, false><<<nblk, RS_THREADS, 0, s>>>(ks, nullptr, kd, nullptr, n, 8 * pass, nblk, off.p);
        BEM_CHECK_LAUNCH();
        ks = kd;
        vs = vd;
    }
    BEM_CUDA(cudaStreamSynchronize(s));  // the buffers are released on return
}

void radix_sort_u64(const uint64_t *k_in, const int *v_in, uint64_t *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s) {
    radix_sort<unsigned long long>(reinterpret_cast<const unsigned long long *>(k_in), v_in,
                                   reinterpret_cast<unsigned long long *>(k_out), v_out, n, bits, s);
}

void radix_sort_u32(const uint32_t *k_in, const int *v_in, uint32_t *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s) {
    radix_sort<unsigned int>(reinterpret_cast<const unsigned int *>(k_in), v_in,
                             reinterpret_cast<unsigned int *>(k_out), v_out, n, bits, s);
}

// --------------------------------------------------------------- unique
__global__ void k_uniq_flags(const uint64_t *key, int64_t n, int *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

__global__ void k_uniq_write(const uint64_t *key, const int *flag, const int *pos, int64_t n, uint64_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = key[i];
}

int64_t unique_sorted_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    DArray<int> flag, pos;
    flag.alloc(n);
    pos.alloc(n);
    k_uniq_flags<<<cdiv(n, 256), 256, 0, s>>>(in, n, flag.p);
    BEM_CHECK_LAUNCH();
    scan_exclusive_i32(flag.p, pos.p, n, s);
    k_uniq_write<<<cdiv(n, 256), 256, 0, s>>>(in, flag.p, pos.p, n, out);
    BEM_CHECK_LAUNCH();
    int last_pos = 0, last_flag = 0;
    BEM_CUDA(cudaMemcpyAsync(&last_pos, pos.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaMemcpyAsync(&last_flag, flag.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    return (int64_t)last_pos + last_flag;
}

}  // namespace bem
