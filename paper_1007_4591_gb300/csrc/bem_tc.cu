// M2L translations on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The M2L step of the downward sweep (Sec. 2.3) is, for every offset class
// o of the interaction list, the dense product L_t += T_o M_s over all pairs
// (t, s) with that offset: with the pairs of one class gathered as columns
// this is a GEMM  D[128 x 64] = T_o[128 x 128] . B[128 x 64]  ((p+1)^2 = 121
// coefficients padded to 128; p <= 10).  It runs as tcgen05.mma kind::tf32
// with the 3xTF32 split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (tf32 keeps
// 11 significant bits; the split recovers FP32-level products), operands in
// shared memory in the canonical K-major layout without swizzle (8 x 16-byte
// core matrices, K-adjacent cores 128 B apart, 8-row groups 4 KB apart), the
// accumulator in tensor memory.  One elected thread issues the 48 MMAs of a
// chunk and commits them to an mbarrier; the four warps then read their 32
// TMEM lanes (one output coefficient per lane) and add them into the local
// expansions with coalesced atomics.  Every wait is bounded: on timeout the
// kernel raises an error flag, waits once more (bounded) for its MMAs and
// frees its tensor memory before returning.
#include <cstring>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

constexpr int TC_BN = 32;          // pairs per MMA tile (N); a 64-pair chunk is two tiles
constexpr int TC_K = 128;          // padded coefficients (K and M)
constexpr int TC_TMEM_COLS = 128;  // allocated columns (two 32-column accumulators, power of two)
constexpr int TC_CHUNKS_PER_CTA = 16;
constexpr long long TC_WAIT_CYCLES = 2000000000ll;  // about one second of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K-adjacent core matrices), stride byte offset (8-row groups),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, N = 32, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > TC_WAIT_CYCLES) return false;
    return true;
}

// element (row, k) of a K-major 128-column tile in core-matrix order (floats)
__host__ __device__ __forceinline__ int tc_off(int row, int k) {
    return (row >> 3) * (TC_K / 4) * 32 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// Warp roles of the pipelined kernel.
constexpr int TC_NS = 3;                       // shared B stages
constexpr int TC_ND = 4;                       // TMEM accumulators of TC_BN columns
constexpr int TC_WARP_MMA = 0;                 // lane 0 issues the MMAs
constexpr int TC_WARP_EPI0 = 1;                // warps 1..4: epilogue (TMEM lane quadrant = warp % 4)
constexpr int TC_WARP_PROD0 = 5;               // warps 5..8: gather of B
constexpr int TC_NPROD = 4 * 32, TC_NEPI = 4 * 32;
constexpr int TC_THREADS = 9 * 32;

// Work item: (offset class, first 64-pair chunk, number of chunks); a
// 64-pair chunk is two tiles of TC_BN = 32 pairs.  Pipeline: producers fill
// B stage t % 3 (mbarrier fullB), the MMA thread waits for it and for the
// accumulator t % 4 to be drained (emptyD), issues the 48 MMAs of the tile
// and commits twice (emptyB: the stage may be refilled; fullD: the
// accumulator is ready); the epilogue warps wait for fullD, read their TMEM
// lanes, release the accumulator (emptyD) and scatter with atomics.
__global__ void __launch_bounds__(TC_THREADS, 1)
k_m2l_tc(const float *__restrict__ Ahi_all, const float *__restrict__ Alo_all,
         const int4 *__restrict__ super, const int4 *__restrict__ chunks,
         const int *__restrict__ p_out, const int *__restrict__ p_in, int nc, int cs,
         const float *__restrict__ Min, float *__restrict__ Lout, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float *Ahi = reinterpret_cast<float *>(smraw);
    float *Alo = Ahi + TC_K * TC_K;
    float *Bbuf = Alo + TC_K * TC_K;  // [TC_NS][hi, lo][TC_BN * TC_K]
    __shared__ __align__(8) uint64_t fullB[TC_NS], emptyB[TC_NS], fullD[TC_ND], emptyD[TC_ND];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 sc = super[blockIdx.x];
    const int ntile = 2 * sc.z;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < TC_NS; ++i) {
            mbar_init(smem_u32(&fullB[i]), TC_NPROD);
            mbar_init(smem_u32(&emptyB[i]), 1);
        }
        for (int i = 0; i < TC_ND; ++i) {
            mbar_init(smem_u32(&fullD[i]), 1);
            mbar_init(smem_u32(&emptyD[i]), TC_NEPI);
        }
        s_fail = 0;
    }
    {  // the operator of this offset class (hi, lo), asynchronous 16-byte copies
        const char *gh = reinterpret_cast<const char *>(Ahi_all + (size_t)sc.x * TC_K * TC_K);
        const char *gl = reinterpret_cast<const char *>(Alo_all + (size_t)sc.x * TC_K * TC_K);
        const uint32_t sh = smem_u32(Ahi), sl = smem_u32(Alo);
        for (int i = tid; i < TC_K * TC_K / 4; i += TC_THREADS) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sh + 16u * i), "l"(gh + 16 * (size_t)i));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sl + 16u * i), "l"(gl + 16 * (size_t)i));
        }
        asm volatile("cp.async.commit_group;");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = s_tmem;

    if (warp >= TC_WARP_PROD0) {
        // ---------------- producers: gather tile t into stage t % TC_NS
        const int ptid = tid - TC_WARP_PROD0 * 32;
        for (int t = 0; t < ntile; ++t) {
            const int st = t % TC_NS, k = t / TC_NS;
            if (k >= 1 && !mbar_wait_bounded(smem_u32(&emptyB[st]), (uint32_t)((k - 1) & 1))) {
                atomicExch(err, 1);
                s_fail = 1;
                break;
            }
            const int4 ch = chunks[sc.y + (t >> 1)];
            const int j0 = 32 * (t & 1);
            float *Bhi = Bbuf + (size_t)st * 2 * TC_BN * TC_K, *Blo = Bhi + TC_BN * TC_K;
            constexpr int PER = TC_BN * (TC_K / 4) / TC_NPROD;  // float4 groups per producer
            float4 v[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int e = ptid + TC_NPROD * u;
                const int n = ((e >> 8) << 3) | (e & 7), k4 = (e >> 3) & 31;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j0 + n < ch.z && 4 * k4 < nc) {
                    const int src = p_in[ch.y + j0 + n];
                    v[u] = __ldg(reinterpret_cast<const float4 *>(Min + (size_t)src * cs + 4 * k4));
                }
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int e = ptid + TC_NPROD * u;
                const int n = ((e >> 8) << 3) | (e & 7), k4 = (e >> 3) & 31;
                float w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                float4 hi, lo;
                float *hp = &hi.x, *lp = &lo.x;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x = (4 * k4 + q < nc) ? w[q] : 0.f;  // the row's padding is not data
                    const uint32_t h = to_tf32(x);
                    hp[q] = __uint_as_float(h);
                    lp[q] = __uint_as_float(to_tf32(x - __uint_as_float(h)));
                }
                const int off = tc_off(n, 4 * k4);
                *reinterpret_cast<float4 *>(Bhi + off) = hi;
                *reinterpret_cast<float4 *>(Blo + off) = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&fullB[st]));
        }
    } else if (warp == TC_WARP_MMA) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
            const uint32_t SBO = (TC_K / 4) * 128, LBO = 128;
            for (int t = 0; t < ntile; ++t) {
                const int st = t % TC_NS, k = t / TC_NS;
                const int d = t % TC_ND, jd = t / TC_ND;
                bool ok = mbar_wait_bounded(smem_u32(&fullB[st]), (uint32_t)(k & 1));
                if (ok && jd >= 1) ok = mbar_wait_bounded(smem_u32(&emptyD[d]), (uint32_t)((jd - 1) & 1));
                if (!ok) {
                    atomicExch(err, 1);
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const float *Bhi = Bbuf + (size_t)st * 2 * TC_BN * TC_K, *Blo = Bhi + TC_BN * TC_K;
                const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Blo);
                const uint32_t dt = tm + (uint32_t)(d * TC_BN);
#pragma unroll 1
                for (int ks = 0; ks < TC_K / 8; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 2 * LBO;
                    const uint64_t dah = tc_desc(ah + ko, LBO, SBO), dal = tc_desc(al + ko, LBO, SBO);
                    const uint64_t dbh = tc_desc(bh + ko, LBO, SBO), dbl = tc_desc(bl + ko, LBO, SBO);
                    tc_mma(dt, dah, dbh, ks > 0 ? 1u : 0u);
                    tc_mma(dt, dah, dbl, 1u);
                    tc_mma(dt, dal, dbh, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&emptyB[st]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&fullD[d]))
                             : "memory");
            }
        }
    } else {
        // ---------------- epilogue: TMEM lane quadrant (warp % 4), 32 pairs per tile
        const int quad = warp & 3;
        const int row = 32 * quad + lane;
        for (int t = 0; t < ntile; ++t) {
            const int d = t % TC_ND, jd = t / TC_ND;
            if (!mbar_wait_bounded(smem_u32(&fullD[d]), (uint32_t)(jd & 1))) {
                atomicExch(err, 1);
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t r[TC_BN];
#pragma unroll
            for (int cg = 0; cg < TC_BN; cg += 16) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[cg + 0]), "=r"(r[cg + 1]), "=r"(r[cg + 2]), "=r"(r[cg + 3]), "=r"(r[cg + 4]),
                      "=r"(r[cg + 5]), "=r"(r[cg + 6]), "=r"(r[cg + 7]), "=r"(r[cg + 8]), "=r"(r[cg + 9]),
                      "=r"(r[cg + 10]), "=r"(r[cg + 11]), "=r"(r[cg + 12]), "=r"(r[cg + 13]),
                      "=r"(r[cg + 14]), "=r"(r[cg + 15])
                    : "r"(tm + ((uint32_t)(32 * quad) << 16) + (uint32_t)(d * TC_BN + cg)));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_u32(&emptyD[d]));
            const int4 ch = chunks[sc.y + (t >> 1)];
            const int j0 = 32 * (t & 1);
            const int cnt = min(TC_BN, ch.z - j0);
            if (row < nc) {
#pragma unroll
                for (int j = 0; j < TC_BN; ++j)
                    if (j < cnt) atomicAdd(Lout + (size_t)p_out[ch.y + j0 + j] * cs + row, __uint_as_float(r[j]));
            }
        }
    }
    // before the CTA's shared memory and tensor memory go away, every commit
    // arrival must have landed: the MMA thread waits (bounded) for the last
    // completion of each B stage and of the last accumulator
    if (warp == TC_WARP_MMA && lane == 0 && ntile > 0) {
        for (int st = 0; st < TC_NS && st < ntile; ++st) {
            const int t = st + ((ntile - 1 - st) / TC_NS) * TC_NS;  // last tile on stage st
            mbar_wait_bounded(smem_u32(&emptyB[st]), (uint32_t)((t / TC_NS) & 1));
        }
        const int t = ntile - 1;
        mbar_wait_bounded(smem_u32(&fullD[t % TC_ND]), (uint32_t)((t / TC_ND) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------- host side
static inline float host_tf32(float x) {
    // round to nearest (ties away from zero) keeping 10 explicit mantissa bits
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return x;
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// hi/lo operator tiles in core order from the column-major double operators
void build_tc_tables(int p, const std::vector<double> &om2l, int nops, std::vector<float> &hi,
                     std::vector<float> &lo) {
    const int nc = (p + 1) * (p + 1);
    hi.assign((size_t)nops * TC_K * TC_K, 0.f);
    lo.assign((size_t)nops * TC_K * TC_K, 0.f);
    for (int o = 0; o < nops; ++o) {
        const double *T = &om2l[(size_t)o * nc * nc];
        float *H = &hi[(size_t)o * TC_K * TC_K], *L = &lo[(size_t)o * TC_K * TC_K];
        for (int row = 0; row < nc; ++row)
            for (int k = 0; k < nc; ++k) {
                const float x = (float)T[(size_t)k * nc + row];
                const float h = host_tf32(x);
                H[tc_off(row, k)] = h;
                L[tc_off(row, k)] = host_tf32(x - h);
            }
    }
}

bool tc_m2l_available(const Mesh &m) {
    return m.opt.precision == BEM_MIXED && (m.opt.p + 1) * (m.opt.p + 1) <= TC_K;
}

size_t tc_smem_bytes() { return (size_t)(2 * TC_K * TC_K + 2 * TC_NS * TC_BN * TC_K) * sizeof(float); }

// super-chunks: up to TC_CHUNKS_PER_CTA consecutive M2L chunks of one offset class
void build_tc_super(Tree &t, const std::vector<int4> &chunks_m2l, cudaStream_t s) {
    std::vector<int4> sup;
    int i = 0;
    const int n = (int)chunks_m2l.size();
    while (i < n) {
        int j = i + 1;
        while (j < n && j - i < TC_CHUNKS_PER_CTA && chunks_m2l[j].x == chunks_m2l[i].x) ++j;
        sup.push_back(make_int4(chunks_m2l[i].x, i, j - i, 0));
        i = j;
    }
    t.tc_super.alloc(sup.size());
    t.tc_nsuper = (int)sup.size();
    if (!sup.empty())
        BEM_CUDA(cudaMemcpyAsync(t.tc_super.p, sup.data(), sup.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
}

void m2l_tc(Mesh &m, const Tree &t, const float *M, float *L) {
    if (t.tc_nsuper == 0) return;
    const size_t sm = tc_smem_bytes();
    ensure_smem_attr(reinterpret_cast<const void *>(k_m2l_tc), sm);
    const int nc = (m.opt.p + 1) * (m.opt.p + 1);
    k_m2l_tc<<<t.tc_nsuper, TC_THREADS, sm, m.stream>>>(m.tab->Tc_hi.p, m.tab->Tc_lo.p, t.tc_super.p,
                                                  t.g_chunk.p + t.m2l_chunk0, t.g_out.p, t.g_in.p, nc,
                                                  cell_stride(m.opt.p), M, L, m.dev_err.p);
    BEM_CHECK_LAUNCH();
}

}  // namespace bem
