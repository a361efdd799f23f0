// M2L translations on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The M2L step of the downward sweep (Sec. 2.3) is, for every offset class
// o of the interaction list, the dense product L_t += T_o M_s over all pairs
// (t, s) with that offset: with the pairs of one class gathered as columns
// this is a GEMM  D[128 x 128] = T_o[128 x 128] . B[128 x 128 pairs]
// ((p+1)^2 = 121 coefficients padded to 128; p <= 10).  It runs as
// tcgen05.mma kind::tf32 with the 3xTF32 split a b ~ a_hi b_hi + a_hi b_lo +
// a_lo b_hi (tf32 keeps 11 significant bits; the split recovers FP32-level
// products).  The operator (A) and the accumulators live in tensor memory;
// the multipoles (B) are staged in shared memory one K-block (32
// coefficients, 128 bytes of a row) at a time in the K-major layout with the
// 128-byte swizzle, so that a warp's copy instruction reads four whole
// 128-byte rows from global memory.  A persistent, warp-specialised kernel
// runs the pairs of one class as a stream of 128-pair tiles (producers, one
// MMA thread, epilogue; see k_m2l_tc).  The epilogue adds each pair's
// local-expansion row into its target cell with vector reductions
// (red.global.add.v4.f32): the targets' local expansions (a few MB) stay in
// L2, which absorbs the reductions at about the rate HBM would take the rows
// (measured 4.9 TB/s against 5.5 TB/s for plain stores), and no per-pair
// buffer is written or read back.  Every wait is bounded: the pipeline waits by
// the mesh's wait budget (bem_set_wait_budget), after which the kernel
// raises an error flag; the last wait for its own MMAs (always about a
// second) comes before it frees its tensor memory and returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

constexpr int TC_BN = 128;           // pairs per MMA tile (N)
constexpr int TC_K = 128;            // padded coefficients (K and M)
constexpr int TC_KB = 32;            // K-block: one 128-byte swizzled row of TF32 values
constexpr int TC_NKB = TC_K / TC_KB; // K-blocks per tile
constexpr int TC_TMEM_COLS = 512;    // A hi [0,128), A lo [128,256), 2 accumulators of 128
constexpr int TC_A_HI = 0, TC_A_LO = 128, TC_D0 = 256;
constexpr int TC_CHUNKS_PER_ITEM = 16;  // 64-pair chunks per work item (8 tiles)
constexpr long long TC_WAIT_CYCLES = 2000000000ll;  // about one second of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address, 8-row groups 1024 B apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128 B).  The leading byte offset is
// not used: one MMA reads 8 TF32 values (32 B) of a row, inside one swizzle
// row; the K-steps inside a K-block advance the start address by 32 B.
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, N = 128, M = 128.
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

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase,
                                                  long long budget = TC_WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// D += A (tensor memory) . B (shared-memory descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

// Warp roles of the pipelined kernel.
constexpr int TC_NS = 5;                       // B stages: one K-block of a tile, hi | lo (32 KB)
constexpr int TC_STAGE_BYTES = 2 * TC_BN * TC_KB * 4;
constexpr int TC_ND = 2;                       // TMEM accumulators of TC_BN columns
constexpr int TC_RING = 16;                    // work items in flight between the roles
constexpr int TC_WARP_MMA = 0;                 // lane 0 issues the MMAs
constexpr int TC_WARP_EPI0 = 1;                // warps 1..4: epilogue (TMEM lane quadrant = warp % 4)
constexpr int TC_WARP_PROD0 = 5;               // warps 5..8: copies of B, operator into TMEM
constexpr int TC_NPROD = 4 * 32, TC_NEPI = 4 * 32;
constexpr int TC_THREADS = 9 * 32;
constexpr int TC_ROWS_PER_PROD = TC_BN * 8 / TC_NPROD;  // rows of a stage per producer thread (8 granules each)

__device__ __forceinline__ void bulk_prefetch_l2(const void *g, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(bytes) : "memory");
}

// The persistent kernel: one CTA per SM takes work items (offset class,
// first pair, number of pairs: up to 8 tiles of 128 pairs) from a global
// counter, largest first.  Tiles are numbered continuously across a CTA's
// items and each tile passes through TC_NKB stages (one per K-block), so the
// pipeline never drains between items:
//  * producers (warps 5-8): the leader fetches the next item, publishes it
//    in a shared ring (mbarrier itemFull) and prefetches its operator into
//    L2; all 128 copy the K-block of the tile's split multipoles into stage
//    g % TC_NS (cp.async: a warp instruction moves four 128-byte rows,
//    written in the 128-byte swizzle; mbarrier fullB).  After the first tile
//    of an item they wait for the last MMA of the previous item (its fullD
//    commit) and write the item's operator into tensor memory (aReady),
//    split from FP32 into its TF32 hi and lo parts on the way.
//  * MMA (warp 0, lane 0): per item waits aReady; per tile waits a free
//    accumulator (emptyD), per K-block its stage (fullB), issues 4 K-steps x
//    3 products with A from tensor memory and commits to emptyB; after the
//    last K-block it commits to fullD.
//  * epilogue (warps 1-4): reads its TMEM lane quadrant, frees the
//    accumulator, transposes the tile into shared memory rows (one local
//    expansion row of cs floats per pair), then the 128 threads add the rows
//    into their target cells of `out`, four coefficients per reduction.
__global__ void __launch_bounds__(TC_THREADS, 1)
k_m2l_tc(const float *__restrict__ A_all,
         const int4 *__restrict__ items, int nitems, int *__restrict__ next_item,
         const int *__restrict__ p_out, const int *__restrict__ p_in, int cs,
         const float *__restrict__ Mtc, float *__restrict__ out, int *__restrict__ err,
         long long budget) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    // 1024-byte aligned base (the 128-byte swizzle repeats every 1024 B)
    unsigned char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sm);
    float *Ct = reinterpret_cast<float *>(sm + (size_t)TC_NS * TC_STAGE_BYTES);  // [TC_BN][cs]
    __shared__ __align__(8) uint64_t fullB[TC_NS], emptyB[TC_NS], fullD[TC_ND], emptyD[TC_ND];
    __shared__ __align__(8) uint64_t aReady, itemFull[TC_RING];
    __shared__ int4 s_item[TC_RING];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
        mbar_init(smem_u32(&aReady), TC_NPROD);
        for (int i = 0; i < TC_RING; ++i) mbar_init(smem_u32(&itemFull[i]), 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = s_tmem;
    // launched as a programmatic dependent of the multipole split: the set-up
    // above overlaps it; the split multipoles, the cleared local expansions
    // and the work counter are read only after this wait
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int ntile_done = 0;  // tiles whose MMAs were all issued (MMA thread)
    int nstage_done = 0; // K-block stages whose MMAs were issued and committed (MMA thread)

    if (warp >= TC_WARP_PROD0) {
        // ---------------- producers
        const int ptid = tid - TC_WARP_PROD0 * 32;
        const int pw = ptid >> 5;                            // producer warp 0..3
        const int quad = warp & 3, row = 32 * quad + lane;  // TMEM lane of this thread
        const int gq = lane & 7, r4 = lane >> 3;            // 16-byte granule, row within a group of 4
        // every wait is made warp-uniform (__all_sync) and every item starts with
        // a vote of all producers, so that on a timeout they leave together
        bool fail = false;
        int t = 0;
        for (int i = 0;; ++i) {
            const int slot = i % TC_RING;
            uint32_t all_ok;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.eq.u32 p, %1, 0;\n bar.red.and.pred q, 2, %2, p;\n"
                " selp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(all_ok)
                : "r"((uint32_t)fail), "n"(TC_NPROD));
            if (!all_ok) break;
            if (ptid == 0) {
                const int idx = atomicAdd(next_item, 1);
                const int4 it = idx < nitems ? items[idx] : make_int4(-1, 0, 0, 0);
                if (it.x >= 0) {
                    bulk_prefetch_l2(A_all + (size_t)it.x * TC_K * TC_K, TC_K * TC_K * 4);
                }
                s_item[slot] = it;
                mbar_arrive(smem_u32(&itemFull[slot]));
            }
            asm volatile("bar.sync 2, %0;" ::"n"(TC_NPROD) : "memory");
            const int4 sc = s_item[slot];
            if (sc.x < 0) break;
            const int ntl = (sc.z + TC_BN - 1) / TC_BN;
            // source cells of the tile rows this thread copies: n = 32 pw + 4 v + r4
            auto load_srcs = [&](int c, int *dst) {
                const int y = sc.y + TC_BN * c, z = min(TC_BN, sc.z - TC_BN * c);
#pragma unroll
                for (int v = 0; v < TC_ROWS_PER_PROD; ++v) {
                    const int n = 32 * pw + 4 * v + r4;
                    dst[v] = (n < z) ? p_in[y + n] : -1;
                }
            };
            int srcs[TC_ROWS_PER_PROD], nxt[TC_ROWS_PER_PROD];
            load_srcs(0, srcs);
            for (int c = 0; c < ntl; ++c, ++t) {
                if (c + 1 < ntl) load_srcs(c + 1, nxt);
                for (int kb = 0; kb < TC_NKB && !fail; ++kb) {
                    const int g = TC_NKB * t + kb;
                    const int st = g % TC_NS, k = g / TC_NS;
                    const bool okB = __all_sync(0xffffffffu, k < 1 || mbar_wait_bounded(smem_u32(&emptyB[st]),
                                                                                       (uint32_t)((k - 1) & 1), budget));
                    if (!okB) {
                        atomicExch(err, 1);
                        fail = true;
                        break;
                    }
                    const uint32_t bh = sbase + (uint32_t)(st * TC_STAGE_BYTES);
                    const uint32_t bl = bh + TC_BN * TC_KB * 4;
#pragma unroll
                    for (int v = 0; v < TC_ROWS_PER_PROD; ++v) {
                        const int n = 32 * pw + 4 * v + r4;
                        const int src = srcs[v];
                        const float *gsrc = Mtc + (size_t)(src >= 0 ? src : 0) * 2 * TC_K + TC_KB * kb + 4 * gq;
                        const uint32_t nb = src >= 0 ? 16u : 0u;  // 0: zero-fill (padding rows)
                        const uint32_t off = (uint32_t)(n * 128 + ((gq ^ (n & 7)) << 4));
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(bh + off), "l"(gsrc), "r"(nb));
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(bl + off), "l"(gsrc + TC_K), "r"(nb));
                    }
                    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&fullB[st])) : "memory");
                }
                if (fail) break;
                if (c == 0) {
                    // the item's operator into tensor memory, once the previous
                    // item's MMAs (which read the old one) have completed
                    const int tp = t - 1;
                    const bool okA = __all_sync(0xffffffffu, t < 1 || mbar_wait_bounded(smem_u32(&fullD[tp % TC_ND]),
                                                                                       (uint32_t)((tp / TC_ND) & 1), budget));
                    if (!okA) {
                        atomicExch(err, 1);
                        fail = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    // operator layout [k / 4][row][k % 4]: the warp's rows read 512
                    // contiguous bytes per load; 32 coefficients at a time, each
                    // split into its TF32 hi part and the TF32 rest (the 3xTF32
                    // operands) and stored to both halves of the operator's columns
                    const float4 *ga = reinterpret_cast<const float4 *>(A_all + (size_t)sc.x * TC_K * TC_K) + row;
#pragma unroll 1
                    for (int part = 0; part < 4; ++part) {
                        const float4 *gp = ga + part * 8 * TC_K;
                        uint32_t vh[32], vl[32];
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            const float4 f = __ldg(gp + (q >> 2) * TC_K);
                            const float x[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                vh[q + e] = to_tf32(x[e]);
                                vl[q + e] = to_tf32(x[e] - __uint_as_float(vh[q + e]));
                            }
                        }
#pragma unroll
                        for (int hl = 0; hl < 2; ++hl) {
                            const uint32_t *v = hl ? vl : vh;
                            asm volatile(
                                "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                                "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(
                                    tm + ((uint32_t)(32 * quad) << 16) + (uint32_t)(hl ? TC_A_LO : TC_A_HI) +
                                    (uint32_t)(32 * part)),
                                "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                                "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]),
                                "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]),
                                "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
                                "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]));
                        }
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(smem_u32(&aReady));
                }
#pragma unroll
                for (int v = 0; v < TC_ROWS_PER_PROD; ++v) srcs[v] = nxt[v];
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == TC_WARP_MMA) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            bool fail = false;
            int t = 0;
            for (int i = 0; !fail; ++i) {
                const int slot = i % TC_RING;
                if (!mbar_wait_bounded(smem_u32(&itemFull[slot]), (uint32_t)((i / TC_RING) & 1), budget)) {
                    atomicExch(err, 1);
                    break;
                }
                const int4 sc = s_item[slot];
                if (sc.x < 0) break;
                if (!mbar_wait_bounded(smem_u32(&aReady), (uint32_t)(i & 1), budget)) {
                    atomicExch(err, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int ntl = (sc.z + TC_BN - 1) / TC_BN;
                for (int c = 0; c < ntl && !fail; ++c, ++t) {
                    const int d = t % TC_ND, jd = t / TC_ND;
                    if (jd >= 1 && !mbar_wait_bounded(smem_u32(&emptyD[d]), (uint32_t)((jd - 1) & 1), budget)) {
                        atomicExch(err, 1);
                        fail = true;
                        break;
                    }
                    const uint32_t dt = tm + (uint32_t)(TC_D0 + d * TC_BN);
                    for (int kb = 0; kb < TC_NKB; ++kb) {
                        const int g = TC_NKB * t + kb;
                        const int st = g % TC_NS, k = g / TC_NS;
                        if (!mbar_wait_bounded(smem_u32(&fullB[st]), (uint32_t)(k & 1), budget)) {
                            atomicExch(err, 1);
                            fail = true;
                            break;
                        }
                        // the stage was written by cp.async (generic proxy): order it before
                        // the tensor core's (async proxy) reads
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t bh = sbase + (uint32_t)(st * TC_STAGE_BYTES);
                        const uint32_t bl = bh + TC_BN * TC_KB * 4;
#pragma unroll
                        for (int ks = 0; ks < TC_KB / 8; ++ks) {
                            const uint64_t dbh = tc_desc_sw128(bh + 32u * ks), dbl = tc_desc_sw128(bl + 32u * ks);
                            const uint32_t kc = (uint32_t)(TC_KB * kb + 8 * ks);
                            tc_mma_ts(dt, tm + TC_A_HI + kc, dbh, (kb | ks) ? 1u : 0u);
                            tc_mma_ts(dt, tm + TC_A_HI + kc, dbl, 1u);
                            tc_mma_ts(dt, tm + TC_A_LO + kc, dbh, 1u);
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         smem_u32(&emptyB[st]))
                                     : "memory");
                        nstage_done = g + 1;
                    }
                    if (fail) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&fullD[d]))
                                 : "memory");
                }
            }
            ntile_done = t;
        }
    } else {
        // ---------------- epilogue: TMEM lane quadrant (warp % 4), 128 pairs per tile
        const int quad = warp & 3;
        const int row = 32 * quad + lane;
        const int etid = tid - TC_WARP_EPI0 * 32;  // 0 .. TC_NEPI - 1
        __shared__ int s_tgt[TC_BN];               // target cells of the tile's pairs
        bool fail = false;
        int t = 0;
        for (int i = 0; !fail; ++i) {
            const int slot = i % TC_RING;
            const bool okI = mbar_wait_bounded(smem_u32(&itemFull[slot]), (uint32_t)((i / TC_RING) & 1), budget);
            uint32_t all_ok;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
                " selp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(all_ok)
                : "r"((uint32_t)okI), "n"(TC_NEPI));
            if (!all_ok) {
                atomicExch(err, 1);
                break;
            }
            const int4 sc = s_item[slot];
            if (sc.x < 0) break;
            const int ntl = (sc.z + TC_BN - 1) / TC_BN;
            for (int c = 0; c < ntl; ++c, ++t) {
                const int d = t % TC_ND, jd = t / TC_ND;
                const bool ok = mbar_wait_bounded(smem_u32(&fullD[d]), (uint32_t)(jd & 1), budget);
                // the four epilogue warps leave together (they meet at named barriers below)
                asm volatile(
                    "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
                    " selp.u32 %0, 1, 0, q;\n}\n"
                    : "=r"(all_ok)
                    : "r"((uint32_t)ok), "n"(TC_NEPI));
                if (!all_ok) {
                    atomicExch(err, 1);
                    fail = true;
                    break;
                }
                // every thread has left the previous tile's reductions (Ct, s_tgt free)
                asm volatile("bar.sync 1, %0;" ::"n"(TC_NEPI) : "memory");
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int y = sc.y + TC_BN * c, z = min(TC_BN, sc.z - TC_BN * c);
                if (etid < z) s_tgt[etid] = p_out[y + etid];
#pragma unroll 1
                for (int cg = 0; cg < TC_BN; cg += 32) {
                    uint32_t r[32];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                        : "r"(tm + ((uint32_t)(32 * quad) << 16) + (uint32_t)(TC_D0 + d * TC_BN + cg)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row < cs) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) Ct[(cg + j) * cs + row] = __uint_as_float(r[j]);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(smem_u32(&emptyD[d]));
                asm volatile("bar.sync 1, %0;" ::"n"(TC_NEPI) : "memory");
                // every pair's row added into its target cell, four coefficients per
                // vector reduction, spread over the epilogue threads
                const int q4 = cs >> 2;
                for (int idx = etid; idx < z * q4; idx += TC_NEPI) {
                    const int j = idx / q4, q = idx - j * q4;
                    const float4 v = *reinterpret_cast<const float4 *>(Ct + j * cs + 4 * q);
                    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(out + (size_t)s_tgt[j] * cs + 4 * q),
                                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                                 : "memory");
                }
            }
        }
    }
    // before the CTA's shared memory and tensor memory go away, every commit
    // arrival must have landed: the MMA thread waits (bounded) for the last
    // completion of each B stage (which follows all MMAs issued before it,
    // also those of a tile left unfinished by a failed wait) and of the last
    // accumulator
    if (warp == TC_WARP_MMA && lane == 0 && nstage_done > 0) {
        const int ng = nstage_done;
        for (int st = 0; st < TC_NS && st < ng; ++st) {
            const int g = st + ((ng - 1 - st) / TC_NS) * TC_NS;  // last stage use on st
            mbar_wait_bounded(smem_u32(&emptyB[st]), (uint32_t)((g / TC_NS) & 1));
        }
        if (ntile_done > 0) {
            const int t = ntile_done - 1;
            mbar_wait_bounded(smem_u32(&fullD[t % TC_ND]), (uint32_t)((t / TC_ND) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------- host side
// The M2L operators in FP32, [offset][k / 4][row = output coefficient][k % 4]
// (k = input coefficient), zero-padded to 128 x 128: the kernel writes row r
// into tensor-memory lane r (its TF32 hi and lo parts), and the 32 rows of a
// warp read 4 consecutive coefficients each from 512 contiguous bytes
void build_tc_tables(int p, const std::vector<double> &om2l, int nops, std::vector<float> &op) {
    const int nc = (p + 1) * (p + 1);
    op.assign((size_t)nops * TC_K * TC_K, 0.f);
    for (int o = 0; o < nops; ++o) {
        const double *T = &om2l[(size_t)o * nc * nc];
        float *A = &op[(size_t)o * TC_K * TC_K];
        for (int row = 0; row < nc; ++row)
            for (int k = 0; k < nc; ++k)
                A[((size_t)(k >> 2) * TC_K + row) * 4 + (k & 3)] = (float)T[(size_t)k * nc + row];
    }
}

bool tc_m2l_available(const Mesh &m) {
    return m.opt.precision == BEM_MIXED && (m.opt.p + 1) * (m.opt.p + 1) <= TC_K;
}

// dynamic shared memory: alignment slack, the B stages, the transposed tile
size_t tc_smem_bytes() { return 1024 + (size_t)TC_NS * TC_STAGE_BYTES + (size_t)TC_BN * TC_K * sizeof(float); }

// Work items of the persistent kernel: (offset class, first pair, number of
// pairs), up to TC_CHUNKS_PER_ITEM consecutive 64-pair chunks of one class
// (tiles of 128 pairs), largest first.
void build_tc_super(Tree &t, const std::vector<int4> &chunks_m2l, cudaStream_t s) {
    std::vector<int4> sup;
    int i = 0;
    const int n = (int)chunks_m2l.size();
    while (i < n) {  // chunks of one class cover consecutive pairs
        int j = i + 1, np = chunks_m2l[i].z;
        while (j < n && j - i < TC_CHUNKS_PER_ITEM && chunks_m2l[j].x == chunks_m2l[i].x) np += chunks_m2l[j++].z;
        sup.push_back(make_int4(chunks_m2l[i].x, chunks_m2l[i].y, np, 0));
        i = j;
    }
    std::stable_sort(sup.begin(), sup.end(), [](const int4 &a, const int4 &b) { return a.z > b.z; });
    t.tc_super.alloc(sup.size());
    t.tc_nsuper = (int)sup.size();
    if (!sup.empty())
        BEM_CUDA(cudaMemcpyAsync(t.tc_super.p, sup.data(), sup.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
}

// hi/lo TF32 split of the multipoles of the M2L sources (cells of levels
// >= 2), rows of 2 x 128 floats: hi | lo, zero beyond (p+1)^2.  One thread
// per 4 coefficients of a cell (16-byte loads and stores; cs is a multiple
// of 4, and a group at or past cs is not read).
__global__ void k_split_m(const float *M, int first, int ncell, int nc, int cs, float *Mtc) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the M2L kernel may start its set-up
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t c = first + (i >> 5);
    const int k0 = 4 * (int)(i & 31);
    if (c >= ncell) return;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k0 < cs) x = *reinterpret_cast<const float4 *>(M + c * cs + k0);
    float v[4] = {x.x, x.y, x.z, x.w};
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (k0 + e >= nc) v[e] = 0.f;
        const uint32_t t = to_tf32(v[e]);
        h[e] = __uint_as_float(t);
        l[e] = __uint_as_float(to_tf32(v[e] - h[e]));
    }
    float *row = Mtc + c * 2 * TC_K;
    *reinterpret_cast<float4 *>(row + k0) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(row + TC_K + k0) = make_float4(l[0], l[1], l[2], l[3]);
}

// L (levels >= 2) = sum over the M2L pairs of T_o M_s: L cleared, the
// multipoles split hi | lo, then the persistent kernel adds every pair's row
// into its target.
void m2l_tc(Mesh &m, const Tree &t, const float *M, float *L, bool timed) {
    const Tables &tb = tables_for(m, t);
    const int nc = (m.opt.p + 1) * (m.opt.p + 1);
    const int cs = cell_stride(m.opt.p);
    const int first = t.lvl_off[2];
    BEM_CUDA(cudaMemsetAsync(L + (size_t)first * cs, 0, (size_t)(t.ncell - first) * cs * sizeof(float), m.stream));
    if (t.tc_nsuper == 0) return;
    if (m.Mtc.n < (size_t)t.ncell * 2 * TC_K) throw Error(BEM_ECUDA, "tensor-core staging buffer too small");
    const bool tk = timed && m.tm.on && m.tm.kev[0];
    auto kev = [&](int k) {
        if (tk) BEM_CUDA(cudaEventRecord(m.tm.kev[k], m.stream));
    };
    BEM_CUDA(cudaMemsetAsync(m.dev_err.p + 1, 0, sizeof(int), m.stream));  // work-item counter
    kev(0);
    if (cs % 4 != 0) throw Error(BEM_ECUDA, "tensor-core staging: cell stride not a multiple of 4");
    k_split_m<<<cdiv((int64_t)(t.ncell - first) * 32, 256), 256, 0, m.stream>>>(M, first, t.ncell, nc, cs, m.Mtc.p);
    BEM_CHECK_LAUNCH();
    const size_t sm = tc_smem_bytes();
    int dev = 0, nsm = 0;
    BEM_CUDA(cudaGetDevice(&dev));
    BEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(t.tc_nsuper, nsm));
    kev(1);
    ensure_smem_attr(reinterpret_cast<const void *>(k_m2l_tc), sm);
    {
        // programmatic dependent launch after the split (the kernel waits
        // before it reads anything the split or earlier work wrote)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = m.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const float *A = tb.Tc_f.p;
        const int4 *items = t.tc_super.p;
        const int nitems = t.tc_nsuper;
        int *counter = m.dev_err.p + 1, *err = m.dev_err.p;
        const int *po = t.g_out.p, *pi = t.g_in.p;
        const float *Mtc = m.Mtc.p;
        const long long budget = m.wait_budget;
        BEM_CUDA(cudaLaunchKernelEx(&cfg, k_m2l_tc, A, items, nitems, counter, po, pi, cs, Mtc, L, err, budget));
    }
    kev(2);
    kev(3);
}

size_t tc_staging_floats(const Mesh &m) {
    return (size_t)std::max(m.tp.ncell, m.tc.ncell) * 2 * TC_K;
}


}  // namespace bem
