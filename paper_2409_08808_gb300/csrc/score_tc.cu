// Batched scoring E_b = q_b^T J_vv q_b + 2 q_b . phi_fix + E_const on the
// tcgen05 tensor cores (sm_103a): the objective of Eq. 2 evaluated for a whole
// population as one dense contraction Phi = J_vv Q followed by a row-dot.
//
// J is symmetric, so E = sum_{I <= J} q_I^T J'_IJ q_J over 128 x 128 blocks
// with J'_II = J_II and J'_IJ = 2 J_IJ (I < J): half the products.  J' is
// split into T low-precision terms (BF16: J' = J1 + J2 [+ J3], each the BF16
// rounding of the remainder; TF32: hi + lo); doubling is exact in both.
// Charges are small integers and exact in BF16 / TF32, so Q needs no split.
// Persistent grid (one CTA per SM), tiles of 128 sites x 256 configurations
// assigned longest-first by the host; the tile of m-block I runs over the
// k-range from column 128 I.  Two FP32 accumulators live in TMEM (2 x 256
// columns) so the epilogue of one tile overlaps the MMAs of the next.  Every
// k-block stage holds the T J'-tiles (128 x 128 B) and one Q-tile (256 x
// 128 B), loaded by TMA with the 128-byte swizzle; the single MMA thread
// issues T x 4 tcgen05.mma (K = 16 BF16 / 8 TF32) into the tile's accumulator.
// Warp roles: warp 0 lane 0 = TMA producer, warp 1 lane 0 = MMA issuer, warps
// 2-5 = epilogue (warp 2 also owns the TMEM allocation): tcgen05.ld of their 32
// TMEM lanes (= 32 sites), q Phi in FP32, a butterfly transpose-reduce
// across the warp so lane l owns config column l, and the 4 warp sums are added
// in FP64 into partial[m-tile][config].  The linear term 2 q . phi_fix is formed
// in FP64 while Q is built (k_make_qt), and a second tiny kernel adds the
// m-tiles in a fixed order plus the linear term and E_const (deterministic).
// The three kernels of a step are chained as programmatic dependent launches:
// each successor sets itself up while its predecessor drains and waits
// (griddepcontrol.wait) before reading the predecessor's output.
#include <cudaTypedefs.h>

#include <math.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <mutex>
#include <queue>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"

namespace {

constexpr int TC_M = 128;              // sites per tile (TMEM lanes)
constexpr int TC_N = 256;              // configurations per tile (TMEM columns), wide shape
constexpr int TC_NS = 128;             // the narrow shape
constexpr int ROW_BYTES = 128;         // one k-block row: 64 BF16 or 32 FP32
constexpr int A_TILE = TC_M * ROW_BYTES;
constexpr int B_TILE = TC_N * ROW_BYTES;
constexpr long long WAIT_LIMIT = 4000000000LL;   // ~2 s of SM clock

// 2^e as a double for e in the normal range (exact; multiplying by it equals
// ldexp(x, e) whenever the product is normal).
__device__ __forceinline__ double pow2(int e)
{
    return __longlong_as_double((long long)(e + 1023) << 52);
}

template <int T, int TN = TC_N>
struct TcCfg {
    static constexpr int STAGE = T * A_TILE + TN * ROW_BYTES;
    static constexpr int STAGES_RAW = (196 * 1024) / STAGE;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int BAR_BYTES = 256;   // stage barriers, 2 + 2 accumulator barriers, TMEM slot, flag
    static constexpr int SMEM = STAGES * STAGE + 1024 + BAR_BYTES;
};

// One unit of work of the persistent scoring kernels: m-block I (128 sites),
// configuration tile n (TN configurations), k-blocks [kb0, kb1) of the
// symmetric operand's row panel I (its columns run from 128 I; the host may
// split that range into chunks), the partial-sum slot it writes and, in the
// exact form, the digit t.
struct TcTile {
    int I, n, kb0, kb1, slot, t;
};

// Persistent kernel.  CTA c processes the tiles work[work_start[c] ..
// work_start[c+1]) (host LPT schedule, longest first).  Each tile's FP64 row-
// dots go to partial[slot][configuration]; the finishing kernel adds the slots
// in a fixed order (the row-dot is linear in Phi, so a split k-range only adds
// slots).
template <int T, bool TF32, int TN>
__global__ void __launch_bounds__(192, 1)
    k_score_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const TcTile* __restrict__ work, const int* __restrict__ work_start, int Nv_pad,
               const void* __restrict__ qt, int ldq, double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    using Cfg = TcCfg<T, TN>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr int STAGE = Cfg::STAGE;
    constexpr int KE = TF32 ? 32 : 64;          // elements per 128-byte row
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;           // [2] accumulator ready
    uint64_t* tempty = tfull + 2;               // [2] accumulator drained
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    __shared__ float red[4][TN];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w0 = work_start[blockIdx.x], w1 = work_start[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, 2 * TN);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // launched as a dependent of k_make_qt: the set-up above overlaps its tail;
    // Q^T (and the linear term) are read only after it has completed
    goacd::pdl_wait();
    goacd::pdl_trigger();

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int it = 0;
            for (int wi = w0; wi < w1 && !*abort_flag; ++wi) {
                const TcTile tile = work[wi];
                const int m0 = tile.I * TC_M, n0 = tile.n * TN;
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (it >= STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * STAGE;
                    goacd::mbar_arrive_expect_tx(&full[s], STAGE);
#pragma unroll
                    for (int t = 0; t < T; ++t)
                        goacd::tma_load_2d(st + t * A_TILE, &tmA, &full[s], kb * KE, t * Nv_pad + m0);
                    goacd::tma_load_2d(st + T * A_TILE, &tmB, &full[s], kb * KE, n0);
                }
            }
            if (*abort_flag) {
                // every copy this thread started must land before the CTA exits
                for (int k = it - STAGES < 0 ? 0 : it - STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % STAGES], (uint32_t)(k / STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(TF32 ? 2u : 1u, TC_M, TN);
            int it = 0, tl = 0;
            for (int wi = w0; wi < w1; ++wi, ++tl) {
                const TcTile tile = work[wi];
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * TN);
                const int kb0 = tile.kb0;
                for (int kb = kb0; kb < tile.kb1; ++kb, ++it) {
                    if (*abort_flag) break;
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a0 = goacd::smem_u32(smem + s * STAGE);
                    const uint32_t b0 = a0 + T * A_TILE;
#pragma unroll
                    for (int t = 0; t < T; ++t)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = goacd::sdesc_k128(a0 + t * A_TILE + kk * 32);
                            const uint64_t bd = goacd::sdesc_k128(b0 + kk * 32);
                            const uint32_t acc = (kb != kb0 || t != 0 || kk != 0) ? 1u : 0u;
                            if (TF32) goacd::mma_tf32(d_tmem, ad, bd, idesc, acc);
                            else goacd::mma_bf16(d_tmem, ad, bd, idesc, acc);
                        }
                    goacd::mma_commit(&empty[s]);
                }
                goacd::mma_commit(&tfull[acc_i]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int lg = warp & 3;                   // TMEM lane group this warp may access
        const int etid = threadIdx.x - 64;         // 0..127
        int tl = 0;
        for (int wi = w0; wi < w1; ++wi, ++tl) {
            const TcTile tile = work[wi];
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            const int v = tile.I * TC_M + lg * 32 + lane;
            const long n0 = (long)tile.n * TN;
#pragma unroll 1
            for (int c = 0; c < TN / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * TN) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                float val[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long b = n0 + c * 32 + j;
                    float q;
                    if (TF32) q = ((const float*)qt)[b * ldq + v];
                    else q = __bfloat162float(((const __nv_bfloat16*)qt)[b * ldq + v]);
                    val[j] = q * __uint_as_float(r[j]);
                }
                // butterfly transpose-reduce: afterwards lane l holds column l summed over the warp
#pragma unroll
                for (int sft = 16; sft >= 1; sft >>= 1) {
                    const bool up = (lane & sft) != 0;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < sft) {
                            const float send = up ? val[k] : val[k + sft];
                            const float keep = up ? val[k + sft] : val[k];
                            val[k] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
                        }
                }
                red[lg][c * 32 + lane] = val[0];
            }
            // the accumulator may be refilled once every warp's loads have completed
            goacd::tc_fence_before();
            __syncwarp();
            if (lane == 0) goacd::mbar_arrive(&tempty[acc_i]);
            goacd::named_bar_sync(1, 128);
            if (ok)
                for (int col = etid; col < TN; col += 128) {
                    const double ssum =
                        (double)red[0][col] + (double)red[1][col] + (double)red[2][col] + (double)red[3][col];
                    partial[(long)tile.slot * Bpad + n0 + col] = ssum;
                }
            goacd::named_bar_sync(1, 128);
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, 2 * TN);
    }
}

__device__ __forceinline__ float to_tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Phi^T = Q^T J (FP32 out) with real Q, TF32 split of both operands:
// Phi = J_hi Q_hi + J_hi Q_lo + J_lo Q_hi (the lo*lo product is dropped).
// Used by the relaxed-occupation gradient, where q = p . z is not integer.
// Persistent grid (one CTA per SM, 192 threads): warp 0 lane 0 TMA producer,
// warp 1 lane 0 MMA issuer (kind::tf32, M = 128 sites, N = 256
// configurations, K = 8), warps 2-5 epilogue (warp 2 owns TMEM).  Tiles of
// 128 sites x 256 configurations over the whole k-range, dealt round robin
// with the configuration block fastest, so the CTAs of one wave cover every
// configuration block of 19 row panels: each panel's J rows come from DRAM
// once and are shared in L2, and the Q tiles are re-read once per wave.  Each
// stage holds J hi / lo (128 x 16 FP32 each) and Q hi / lo (256 x 16 FP32
// each) in 64-byte-swizzled rows: 48 KB for six MMAs (8 KB in by TMA and
// 12 KB out to the tensor core per MMA, as in the two-term BF16 scoring
// kernel); four stages fit, three of them in flight while the tensor core
// works on the fourth.  Two FP32 accumulators in
// TMEM (2 x 256 columns) let the epilogue of one tile, which writes its 32
// TMEM lanes (sites) to Phi[b][v] coalesced over sites, overlap the MMAs of
// the next.  The padded batch is a multiple of 256.  The tiles that would
// leave the last wave partly idle are split into two k-halves whose epilogues
// add into a zeroed Phi (two FP32 addends onto zero: the same sum in either
// order), so the wave count matches the work.  Odd waves walk the k-range
// backwards: the Q slices the previous wave read last are still in L2 when
// the next wave starts, which saves part of the once-per-wave Q re-read.
constexpr int PT_N = 256;
constexpr int PT_ROW = 64;                    // bytes of one operand row in a stage (16 FP32)
constexpr int PT_KB = PT_ROW / 4;             // k elements per stage
constexpr int PT_A = TC_M * PT_ROW;           // 8 KB
constexpr int PT_B = PT_N * PT_ROW;           // 16 KB
constexpr int PT_STAGE = 2 * PT_A + 2 * PT_B; // 48 KB
constexpr int PT_STAGES = 4;
constexpr int PT_SMEM = PT_STAGES * PT_STAGE + 1024 + 256;

// TMA tile load with an L2 eviction-priority hint (a policy made by createpolicy).
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                 uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(goacd::smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(goacd::smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Shared-memory descriptor of a K-major operand tile with 64-byte rows and the
// 64-byte swizzle (8-row groups 512 bytes apart).
__device__ __forceinline__ uint64_t sdesc_k64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;                // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
    d |= (uint64_t)4 << 61;                         // 64-byte swizzle
    return d;
}

// Work item `it` of k_phi_tc: the first nfull items are whole tiles (m-block,
// configuration block fastest); each later tile is two items, its k-halves.
struct PhiItem {
    int m0, n0, kb0, kb1;
    bool add;
};

__device__ __forceinline__ PhiItem phi_item(int it, int nfull, int nbn, int nkb)
{
    PhiItem w;
    int tile = it, half = -1;
    if (it >= nfull) {
        tile = nfull + (it - nfull) / 2;
        half = (it - nfull) % 2;
    }
    w.m0 = (tile / nbn) * TC_M;
    w.n0 = (tile % nbn) * PT_N;
    w.kb0 = half <= 0 ? 0 : nkb / 2;
    w.kb1 = half == 0 ? nkb / 2 : nkb;
    w.add = half >= 0;
    return w;
}

// F16: the same kernel on kind::f16 with FP16 operands (J scaled per 128-row
// panel I by 2^(15 - e_I) and q by 2^qshift, so that the hi / lo parts stay in
// FP16's range; 32 k-columns per 64-byte row), twice the TF32 rate; the
// epilogue multiplies the tile by 2^(e_I - 15 - qshift) (exact).
template <bool F16>
__global__ void __launch_bounds__(192, 1)
    k_phi_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int nitems, int nfull,
             int nbn, int nkb, int ld, int Bpad, const int* __restrict__ pexp, int qshift, float* __restrict__ Phi,
             int* __restrict__ err)
{
    constexpr int KB = F16 ? 32 : PT_KB;         // k elements per stage (64-byte rows)
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + PT_STAGES * PT_STAGE);
    uint64_t* empty = full + PT_STAGES;
    uint64_t* tfull = empty + PT_STAGES;         // [2] accumulator ready
    uint64_t* tempty = tfull + 2;                // [2] accumulator drained
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < PT_STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, 2 * PT_N);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint64_t pol_j = l2_policy_evict_first(), pol_q = l2_policy_evict_last();
            int it = 0;
            for (int id = blockIdx.x; id < nitems && !*abort_flag; id += gridDim.x) {
                const PhiItem w = phi_item(id, nfull, nbn, nkb);
                const int m0 = w.m0, n0 = w.n0;
                const bool rev = ((id / gridDim.x) & 1) != 0;
                for (int j = 0; j < w.kb1 - w.kb0; ++j, ++it) {
                    const int kb = rev ? w.kb1 - 1 - j : w.kb0 + j;
                    const int s = it % PT_STAGES;
                    const uint32_t use = (uint32_t)(it / PT_STAGES);
                    if (it >= PT_STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * PT_STAGE;
                    goacd::mbar_arrive_expect_tx(&full[s], PT_STAGE);
                    // J's panels stream past (each is read by one wave), Q is read again by every wave:
                    // J's lines go first from L2, Q's last
                    tma_load_2d_hint(st, &tmA, &full[s], kb * KB, m0, pol_j);
                    tma_load_2d_hint(st + PT_A, &tmA, &full[s], kb * KB, ld + m0, pol_j);
                    tma_load_2d_hint(st + 2 * PT_A, &tmB, &full[s], kb * KB, n0, pol_q);
                    tma_load_2d_hint(st + 2 * PT_A + PT_B, &tmB, &full[s], kb * KB, Bpad + n0, pol_q);
                }
            }
            if (*abort_flag)
                for (int k = it - PT_STAGES < 0 ? 0 : it - PT_STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % PT_STAGES], (uint32_t)(k / PT_STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(F16 ? 0u : 2u, TC_M, PT_N);   // FP16 or TF32
            int it = 0, tl = 0;
            for (int id = blockIdx.x; id < nitems; id += gridDim.x, ++tl) {
                const PhiItem w = phi_item(id, nfull, nbn, nkb);
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * PT_N);
                for (int j = 0; j < w.kb1 - w.kb0; ++j, ++it) {
                    if (*abort_flag) break;
                    const int s = it % PT_STAGES;
                    const uint32_t use = (uint32_t)(it / PT_STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a_hi = goacd::smem_u32(smem + s * PT_STAGE);
                    const uint32_t a_lo = a_hi + PT_A;
                    const uint32_t b_hi = a_hi + 2 * PT_A;
                    const uint32_t b_lo = b_hi + PT_B;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {    // K = 8 (TF32) or 16 (FP16) per MMA: 32 bytes of each row
                        const uint32_t off = kk * 32;
                        if constexpr (F16) {
                            goacd::mma_bf16(d_tmem, sdesc_k64(a_hi + off), sdesc_k64(b_hi + off), idesc,
                                            (j != 0 || kk != 0) ? 1u : 0u);
                            goacd::mma_bf16(d_tmem, sdesc_k64(a_hi + off), sdesc_k64(b_lo + off), idesc, 1u);
                            goacd::mma_bf16(d_tmem, sdesc_k64(a_lo + off), sdesc_k64(b_hi + off), idesc, 1u);
                        } else {
                            goacd::mma_tf32(d_tmem, sdesc_k64(a_hi + off), sdesc_k64(b_hi + off), idesc,
                                            (j != 0 || kk != 0) ? 1u : 0u);
                            goacd::mma_tf32(d_tmem, sdesc_k64(a_hi + off), sdesc_k64(b_lo + off), idesc, 1u);
                            goacd::mma_tf32(d_tmem, sdesc_k64(a_lo + off), sdesc_k64(b_hi + off), idesc, 1u);
                        }
                    }
                    goacd::mma_commit(&empty[s]);
                }
                goacd::mma_commit(&tfull[acc_i]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int lg = warp & 3;                   // TMEM lane group this warp may access
        int tl = 0;
        for (int id = blockIdx.x; id < nitems; id += gridDim.x, ++tl) {
            const PhiItem w = phi_item(id, nfull, nbn, nkb);
            const int m0 = w.m0, n0 = w.n0;
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            const int v = m0 + lg * 32 + lane;
            const float sc = F16 ? __int_as_float((pexp[m0 / TC_M] - 15 - qshift + 127) << 23) : 1.0f;
#pragma unroll 1
            for (int c = 0; c < PT_N / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * PT_N) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                if (ok && !w.add) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) Phi[(long)(n0 + c * 32 + j) * ld + v] = __uint_as_float(r[j]) * sc;
                } else if (ok) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        atomicAdd(&Phi[(long)(n0 + c * 32 + j) * ld + v], __uint_as_float(r[j]) * sc);
                }
            }
            goacd::tc_fence_before();
            __syncwarp();
            if (lane == 0) goacd::mbar_arrive(&tempty[acc_i]);
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, 2 * PT_N);
    }
}

// Full (not symmetric) J split in TF32 hi / lo for the Phi-output path.
__global__ void k_split_tf32_full(const double* __restrict__ J, long n, float* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double x = J[e];
        const float hi = to_tf32_rna((float)x);
        out[e] = hi;
        out[n + e] = to_tf32_rna((float)(x - (double)hi));
    }
}

// ---------------------------------------------------------------------------
// Exact form: integer-digit split of the symmetric operand on tcgen05.
// J' (128-block upper triangle as above) is scaled per 128-row panel I by
// 2^-e_I (|J'| < 2^e_I) and written as T signed digits of r bits,
// J'/2^e_I = sum_t a_t 2^-(r-1+rt) + res, a_t in [-2^(r-1), 2^(r-1)] (exact in
// FP16 for r <= 11), |res| <= 2^-rT.  The host picks r = 10, T = 5 (50 bits)
// when 2^9 max|q| Nv_pad < 2^24, else r = 8, T = 6 (48 bits) when
// 2^7 max|q| Nv_pad < 2^24.  Charges are integers after a power-of-two
// scaling and exact in FP16, so every product a_t q and every partial sum over
// <= Nv_pad sites is an integer below 2^24: the FP32 accumulators hold the
// digit sums Phi_t = A_t Q exactly.  A tile is (panel I, 256 configurations,
// digit t): the same M = 128 sites x N = 256 configurations MMA shape, stage
// layout and double-buffered TMEM accumulators as k_score_tc with one term,
// with kind::f16 on FP16 operands.  The epilogue forms P_t,b = sum_i q_bi
// Phi_t,ib exactly in 32-bit integers and stores it as an FP64 integer
// (k_finish_exact scales by 2^(e_I - (r-1) - rt)): when the host's bound
// 32 max|q| max|Phi| < 2^31 holds, each warp sums q Phi over its 32 sites in
// one int32 butterfly and the four warp sums are added in 64 bits; else
// (SPLIT) each accumulator is split into 12-bit halves so that no sum over the
// 128 sites can overflow, at twice the shuffles.
constexpr int EX_STAGE = A_TILE + B_TILE;      // 48 KB (k_phi_exact)
constexpr int EX_STAGES = 4;
constexpr int EX_SMEM = EX_STAGES * EX_STAGE + 1024 + 256;

// Stages of k_score_exact for a tile width: as many as fit in 196 KB, at most 6.
template <int TN>
struct ExCfg {
    static constexpr int STAGE = A_TILE + TN * ROW_BYTES;
    static constexpr int STAGES = (196 * 1024) / STAGE > 6 ? 6 : (196 * 1024) / STAGE;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

// Non-split instances are compiled for at most 168 registers (two blocks' worth; the shared memory
// still admits one) so that k_make_qt's blocks can share the SM while the kernel's prologue runs.
template <int TN, bool SPLIT>
__global__ void __launch_bounds__(192, SPLIT ? 1 : 2)
    k_score_exact(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const TcTile* __restrict__ work, const int* __restrict__ work_start, int ld, int T,
                  const __half* __restrict__ qt, double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int STAGE = ExCfg<TN>::STAGE;
    constexpr int STAGES = ExCfg<TN>::STAGES;
    static_assert(STAGES * STAGE + 1024 + 256 <= ExCfg<TN>::SMEM, "stages exceed the dynamic shared memory");
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;           // [2] accumulator ready
    uint64_t* tempty = tfull + 2;               // [2] accumulator drained
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    __shared__ int red_hi[4][TN], red_lo[4][TN];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w0 = work_start[blockIdx.x], w1 = work_start[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, 2 * TN);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // launched as a dependent of k_make_qt: the set-up above overlaps its tail
    goacd::pdl_wait();
    goacd::pdl_trigger();

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int it = 0;
            for (int wi = w0; wi < w1 && !*abort_flag; ++wi) {
                const TcTile tile = work[wi];
                const int m0 = tile.I * TC_M, n0 = tile.n * TN, t = tile.t;
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (it >= STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * STAGE;
                    goacd::mbar_arrive_expect_tx(&full[s], STAGE);
                    goacd::tma_load_2d(st, &tmA, &full[s], kb * 64, t * ld + m0);
                    goacd::tma_load_2d(st + A_TILE, &tmB, &full[s], kb * 64, n0);
                }
            }
            if (*abort_flag)
                for (int k = it - STAGES < 0 ? 0 : it - STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % STAGES], (uint32_t)(k / STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(0u, TC_M, TN);   // FP16 digits and charges
            int it = 0, tl = 0;
            for (int wi = w0; wi < w1; ++wi, ++tl) {
                const TcTile tile = work[wi];
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * TN);
                const int kb0 = tile.kb0;
                for (int kb = kb0; kb < tile.kb1; ++kb, ++it) {
                    if (*abort_flag) break;
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a0 = goacd::smem_u32(smem + s * STAGE);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        goacd::mma_bf16(d_tmem, goacd::sdesc_k128(a0 + kk * 32),
                                        goacd::sdesc_k128(a0 + A_TILE + kk * 32), idesc,
                                        (kb != kb0 || kk != 0) ? 1u : 0u);
                    goacd::mma_commit(&empty[s]);
                }
                goacd::mma_commit(&tfull[acc_i]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int lg = warp & 3;
        const int etid = threadIdx.x - 64;
        // the charges of this thread's site for the tile's TN configurations, loaded before the
        // tile's accumulator is ready so that the epilogue itself is pure ALU work: int16 pairs when
        // SPLIT (|q| < 1024: the digit width rule keeps 2^7 max|q| Nv_pad < 2^24, Nv_pad >= 128),
        // else int8 quadruples (32 max|q|^2 2^(r-1) Nv_pad < 2^31 with r >= 8 gives |q| < 64), which
        // keeps the register count low enough for k_make_qt's blocks to share the SM
        constexpr int QPW = SPLIT ? 2 : 4;           // charges per 32-bit word
        uint32_t qp[TN / QPW];
        auto load_q = [&](const TcTile& tq) {
            const __half* src = qt + (long)tq.n * TN * ld + tq.I * TC_M + lg * 32 + lane;
#pragma unroll
            for (int j = 0; j < TN / QPW; ++j) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < QPW; ++e) {
                    const int q = __float2int_rn(__half2float(src[(long)(QPW * j + e) * ld]));
                    w |= ((uint32_t)q & (SPLIT ? 0xffffu : 0xffu)) << ((32 / QPW) * e);
                }
                qp[j] = w;
            }
        };
        if (w0 < w1) load_q(work[w0]);
        int tl = 0;
        for (int wi = w0; wi < w1; ++wi, ++tl) {
            const TcTile tile = work[wi];
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            const long n0 = (long)tile.n * TN;
#pragma unroll
            for (int c = 0; c < TN / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * TN) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                int hi[32], lo[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const uint32_t w2 = qp[(c * 32 + j) / QPW];
                    constexpr int QB = 32 / QPW;             // bits per charge
                    const int e = j % QPW;
                    const int q = (int)(w2 << (32 - QB * (e + 1))) >> (32 - QB);   // sign-extended field e
                    const int a = __float2int_rn(__uint_as_float(r[j]));   // |a| < 2^24, exact
                    if (SPLIT) {
                        hi[j] = (a >> 12) * q;
                        lo[j] = (a & 4095) * q;
                    } else {
                        hi[j] = a * q;          // the host checked 32 max|q a| < 2^31
                    }
                }
                // butterfly transpose-reduce: afterwards lane l holds column l summed over the warp
#pragma unroll
                for (int sft = 16; sft >= 1; sft >>= 1) {
                    const bool up = (lane & sft) != 0;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < sft) {
                            const int sh = up ? hi[k] : hi[k + sft], kh = up ? hi[k + sft] : hi[k];
                            hi[k] = kh + __shfl_xor_sync(0xffffffffu, sh, sft);
                            if (SPLIT) {
                                const int sl = up ? lo[k] : lo[k + sft], kl = up ? lo[k + sft] : lo[k];
                                lo[k] = kl + __shfl_xor_sync(0xffffffffu, sl, sft);
                            }
                        }
                }
                red_hi[lg][c * 32 + lane] = hi[0];
                if (SPLIT) red_lo[lg][c * 32 + lane] = lo[0];
            }
            goacd::tc_fence_before();
            __syncwarp();
            if (lane == 0) goacd::mbar_arrive(&tempty[acc_i]);
            if (wi + 1 < w1) load_q(work[wi + 1]);
            goacd::named_bar_sync(1, 128);
            if (ok)
                for (int col = etid; col < TN; col += 128) {
                    double pt;
                    if (SPLIT) {
                        const int sh = red_hi[0][col] + red_hi[1][col] + red_hi[2][col] + red_hi[3][col];
                        const int sl = red_lo[0][col] + red_lo[1][col] + red_lo[2][col] + red_lo[3][col];
                        pt = (double)sh * 4096.0 + (double)sl;
                    } else {
                        pt = (double)((long long)red_hi[0][col] + red_hi[1][col] + red_hi[2][col] + red_hi[3][col]);
                    }
                    partial[((long)tile.slot * T + tile.t) * Bpad + n0 + col] = pt;
                }
            goacd::named_bar_sync(1, 128);
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, 2 * TN);
    }
}

// Exact form on CTA pairs (tcgen05 cta_group::2): a cluster of two CTAs on
// one TPC computes a tile of 256 configurations (128 on each CTA's tensor-
// memory lanes) x one pair-panel of 256 sites (the rows 256 P .. 256 P + 255
// of digit t of J': panels 2P and 2P + 1) with M = 256 MMAs issued by the even
// CTA.  Each CTA loads its own 128 configurations' rows of Q^T (the M half)
// and its panel's 128 digit rows (the N half), 16 KB each per k-block, so a
// CTA's shared memory takes in 32 KB per k-block where the one-CTA kernels
// take 48 KB, and six stages fit where those fit four.  The accumulator row of
// configuration b holds Phi_t,ib for the pair-panel's 256 sites, and the
// epilogue thread that owns it forms P_t,I,b = sum_i q_bi Phi_t,ib over each
// panel's 128 sites by itself, from an int8 copy of Q^T (int16 when the digit
// sums split) that k_make_qt writes beside the FP16 operand: no cross-lane
// reduction and no shared memory.  Each 32-site chunk of products is summed in
// int32 under the same host bound as the one-CTA kernel (32 max|q a| < 2^31),
// the chunks in 64 bits; the split case sums the products in 64 bits directly.
// Pair-panel P covers columns from 256 P, so panel 2P + 1 multiplies one
// 128 x 128 block of zeros (below the diagonal of the symmetric operand).
// Barriers: the even CTA's full[s] counts both CTAs' TMA bytes (the odd CTA's
// loads signal it through its cluster address), the MMA commits arrive on
// empty[s] and tfull[a] of both CTAs, and the eight epilogue warps of the pair
// arrive on the even CTA's tempty[a] as soon as their accumulator rows are
// read.  Every wait is clock-bounded as in the one-CTA kernels; both CTAs
// meet at a cluster barrier before freeing their tensor memory and exiting.
struct PairTile {
    int P, n, kb0, kb1, slot0, slot1, t;    // slot1 < 0: panel 2P + 1 does not exist
};

// Byte e (SPLIT: half-word e) of w, sign-extended: prmt's selector nibbles with
// the top bit set replicate the sign of the selected byte.
template <bool WIDE, int E>
__device__ __forceinline__ int ct_charge(uint32_t w)
{
    constexpr uint32_t lo = WIDE ? 2 * E : E, hi = WIDE ? 2 * E + 1 : E;
    constexpr uint32_t sel = lo | (WIDE ? hi << 4 : (8 | hi) << 4) | ((8 | hi) << 8) | ((8 | hi) << 12);
    int r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(w), "r"(sel));
    return r;
}

constexpr int PX_HN = 128;                              // configurations per CTA's half of the tile
constexpr int PX_STAGE = A_TILE + PX_HN * ROW_BYTES;    // 32 KB
constexpr int PX_STAGES = 6;
constexpr int PX_SMEM = PX_STAGES * PX_STAGE + 1024 + 256;

template <bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
    k_score_exact_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const PairTile* __restrict__ work, const int* __restrict__ work_start, int ld, int T,
                       const void* __restrict__ qi, double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    constexpr int TN = 256;                     // sites per tile: TMEM columns
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + PX_STAGES * PX_STAGE);
    uint64_t* empty = full + PX_STAGES;
    uint64_t* tfull = empty + PX_STAGES;        // [2] accumulator ready
    uint64_t* tempty = tfull + 2;               // [2] accumulator drained (the even CTA's counts both)
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = goacd::cluster_ctarank();
    const int pair = blockIdx.x >> 1;
    const int w0 = work_start[pair], w1 = work_start[pair + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < PX_STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 8);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc_pair(tmem_slot, 2 * TN);
        goacd::tmem_relinquish_pair();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::cluster_sync();                      // the even CTA's barriers exist before the odd one signals them
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    goacd::pdl_wait();
    goacd::pdl_trigger();

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            int it = 0;
            for (int wi = w0; wi < w1 && !*abort_flag; ++wi) {
                const PairTile tile = work[wi];
                // this CTA's 128 configurations (the M half) and its panel's digit rows (the N half)
                const int q0 = tile.n * 256 + (int)rank * PX_HN, j0 = tile.t * ld + (2 * tile.P + (int)rank) * TC_M;
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    const int s = it % PX_STAGES;
                    const uint32_t use = (uint32_t)(it / PX_STAGES);
                    if (it >= PX_STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * PX_STAGE;
                    const uint32_t fbar = goacd::mapa_shared(goacd::smem_u32(&full[s]), 0);
                    if (rank == 0) goacd::mbar_arrive_expect_tx(&full[s], 2 * PX_STAGE);
                    goacd::tma_load_2d_pair(st, &tmA, fbar, kb * 64, q0);
                    goacd::tma_load_2d_pair(st + A_TILE, &tmB, fbar, kb * 64, j0);
                }
            }
            if (*abort_flag && rank == 0)
                // every copy of the pair counted on these barriers must land before the CTAs exit
                for (int k = it - PX_STAGES < 0 ? 0 : it - PX_STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % PX_STAGES], (uint32_t)(k / PX_STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (the even CTA) ----------------
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(0u, 2 * PX_HN, TN);   // FP16, M = 256
            int it = 0, tl = 0;
            for (int wi = w0; wi < w1; ++wi, ++tl) {
                const PairTile tile = work[wi];
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * TN);
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    if (*abort_flag) break;
                    const int s = it % PX_STAGES;
                    const uint32_t use = (uint32_t)(it / PX_STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a0 = goacd::smem_u32(smem + s * PX_STAGE);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        goacd::mma_f16_pair(d_tmem, goacd::sdesc_k128(a0 + kk * 32),
                                            goacd::sdesc_k128(a0 + A_TILE + kk * 32), idesc,
                                            (kb != tile.kb0 || kk != 0) ? 1u : 0u);
                    goacd::mma_commit_pair(&empty[s], 0x3);
                }
                goacd::mma_commit_pair(&tfull[acc_i], 0x3);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 of both CTAs, one configuration per thread ----------------
        const int lg = warp & 3;
        constexpr int QPW = SPLIT ? 2 : 4;          // charges per 32-bit word
        uint32_t qp[TN / QPW];
        auto load_q = [&](const PairTile& tq) {
            const long b = (long)tq.n * 256 + (int)rank * PX_HN + lg * 32 + lane;
            const uint4* src = (const uint4*)((const uint8_t*)qi + (b * ld + 2 * tq.P * TC_M) * (SPLIT ? 2 : 1));
            const bool two = tq.slot1 >= 0;     // else the sites past panel 2P lie outside the row
#pragma unroll
            for (int u = 0; u < TN / QPW / 4; ++u) {
                const uint4 v = (u < TN / QPW / 8 || two) ? __ldg(src + u) : make_uint4(0u, 0u, 0u, 0u);
                qp[4 * u] = v.x;
                qp[4 * u + 1] = v.y;
                qp[4 * u + 2] = v.z;
                qp[4 * u + 3] = v.w;
            }
        };
        if (w0 < w1) load_q(work[w0]);
        int tl = 0;
        for (int wi = w0; wi < w1; ++wi, ++tl) {
            const PairTile tile = work[wi];
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            long long s0 = 0, s1 = 0;               // panels 2P and 2P + 1
#pragma unroll
            for (int c = 0; c < TN / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * TN) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                if (c == TN / 32 - 1) {
                    // the accumulator rows have been read: the MMA may start the tile after next in them
                    goacd::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0) goacd::mbar_arrive(&tempty[acc_i]);
                        else goacd::mbar_arrive_cluster(goacd::mapa_shared(goacd::smem_u32(&tempty[acc_i]), 0));
                    }
                }
                long long cs;
                if constexpr (SPLIT) {
                    cs = 0;
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const uint32_t w = qp[(c * 32 + j) / 2];
                        cs += (long long)__float2int_rn(__uint_as_float(r[j])) * ct_charge<true, 0>(w);
                        cs += (long long)__float2int_rn(__uint_as_float(r[j + 1])) * ct_charge<true, 1>(w);
                    }
                } else {
                    int sum = 0;                    // |a| < 2^24 exact in FP32; 32 max|q a| < 2^31
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const uint32_t w = qp[(c * 32 + j) / 4];
                        sum += __float2int_rn(__uint_as_float(r[j])) * ct_charge<false, 0>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 1])) * ct_charge<false, 1>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 2])) * ct_charge<false, 2>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 3])) * ct_charge<false, 3>(w);
                    }
                    cs = sum;
                }
                if (c < TN / 64) s0 += cs;
                else s1 += cs;
            }
            if (wi + 1 < w1) load_q(work[wi + 1]);
            if (ok) {
                const long b = (long)tile.n * 256 + (int)rank * PX_HN + lg * 32 + lane;
                partial[((long)tile.slot0 * T + tile.t) * Bpad + b] = (double)s0;
                if (tile.slot1 >= 0) partial[((long)tile.slot1 * T + tile.t) * Bpad + b] = (double)s1;
            }
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::cluster_sync();                      // no CTA leaves while its peer may still reach its memory
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc_pair(tmem, 2 * TN);
    }
}

// Split forms (BF16 or TF32 terms) on CTA pairs, laid out as
// k_score_exact_pair: a tile is 256 configurations (128 on each CTA's
// tensor-memory lanes) x one pair-panel of 256 sites, M = 256 MMAs issued by
// the even CTA; each CTA loads its own 128 configurations' rows of Q^T and,
// for each of the T terms of J', its panel's 128 rows (128-byte rows: 64 BF16
// or 32 TF32 k-elements per stage), and the T terms accumulate into the same
// FP32 tile.  The epilogue thread that owns configuration b forms q_b . Phi
// over each panel's 128 sites by itself: per 32-site chunk an FP32 sum of
// q Phi (the charges read from the BF16 or FP32 row of Q^T two chunks ahead,
// one for FP32),
// the chunks added in FP64.  Slots are pair_schedule's (one per panel and
// k-chunk, no digit index).
template <int T>
struct TpCfg {
    static constexpr int STAGE = (1 + T) * A_TILE;                  // Q^T rows, then T x J' rows
    static constexpr int STAGES = (196 * 1024) / STAGE > 6 ? 6 : (196 * 1024) / STAGE;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

// D (+)= A * B^T over the CTA pair, kind::tf32 (operand layout as mma_f16_pair).
__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

template <int T, bool TF32>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
    k_score_tc_pair(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmJ,
                    const PairTile* __restrict__ work, const int* __restrict__ work_start, int ld,
                    const void* __restrict__ qt, double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    using Cfg = TpCfg<T>;
    constexpr int STAGES = Cfg::STAGES, STAGE = Cfg::STAGE;
    constexpr int TN = 256;                     // sites per tile: TMEM columns
    constexpr int KE = TF32 ? 32 : 64;          // k elements per 128-byte row
    constexpr int QB = TF32 ? 4 : 2;            // bytes of one charge in Q^T
    static_assert(STAGES * STAGE + 1024 + 256 <= Cfg::SMEM, "stages exceed the dynamic shared memory");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;           // [2] accumulator ready
    uint64_t* tempty = tfull + 2;               // [2] accumulator drained (the even CTA's counts both)
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = goacd::cluster_ctarank();
    const int pair = blockIdx.x >> 1;
    const int w0 = work_start[pair], w1 = work_start[pair + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 8);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmQ);
        goacd::prefetch_tmap(&tmJ);
    }
    if (warp == 2) {
        goacd::tmem_alloc_pair(tmem_slot, 2 * TN);
        goacd::tmem_relinquish_pair();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::cluster_sync();                      // the even CTA's barriers exist before the odd one signals them
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    goacd::pdl_wait();
    goacd::pdl_trigger();

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            int it = 0;
            for (int wi = w0; wi < w1 && !*abort_flag; ++wi) {
                const PairTile tile = work[wi];
                const int q0 = tile.n * 256 + (int)rank * PX_HN, j0 = (2 * tile.P + (int)rank) * TC_M;
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (it >= STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * STAGE;
                    const uint32_t fbar = goacd::mapa_shared(goacd::smem_u32(&full[s]), 0);
                    if (rank == 0) goacd::mbar_arrive_expect_tx(&full[s], 2 * STAGE);
                    goacd::tma_load_2d_pair(st, &tmQ, fbar, kb * KE, q0);
#pragma unroll
                    for (int t = 0; t < T; ++t)
                        goacd::tma_load_2d_pair(st + (1 + t) * A_TILE, &tmJ, fbar, kb * KE, t * ld + j0);
                }
            }
            if (*abort_flag && rank == 0)
                // every copy of the pair counted on these barriers must land before the CTAs exit
                for (int k = it - STAGES < 0 ? 0 : it - STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % STAGES], (uint32_t)(k / STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (the even CTA) ----------------
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(TF32 ? 2u : 1u, 2 * PX_HN, TN);   // M = 256
            int it = 0, tl = 0;
            for (int wi = w0; wi < w1; ++wi, ++tl) {
                const PairTile tile = work[wi];
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * TN);
                for (int kb = tile.kb0; kb < tile.kb1; ++kb, ++it) {
                    if (*abort_flag) break;
                    const int s = it % STAGES;
                    const uint32_t use = (uint32_t)(it / STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a0 = goacd::smem_u32(smem + s * STAGE);
#pragma unroll
                    for (int t = 0; t < T; ++t)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = goacd::sdesc_k128(a0 + kk * 32);
                            const uint64_t bd = goacd::sdesc_k128(a0 + (1 + t) * A_TILE + kk * 32);
                            const uint32_t acc = (kb != tile.kb0 || t != 0 || kk != 0) ? 1u : 0u;
                            if (TF32) mma_tf32_pair(d_tmem, ad, bd, idesc, acc);
                            else goacd::mma_f16_pair(d_tmem, ad, bd, idesc, acc);
                        }
                    goacd::mma_commit_pair(&empty[s], 0x3);
                }
                goacd::mma_commit_pair(&tfull[acc_i], 0x3);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 of both CTAs, one configuration per thread ----------------
        const int lg = warp & 3;
        constexpr int QW = 32 * QB / 4;             // words of one 32-site chunk's charges
        constexpr int PF = TF32 ? 1 : 2;            // chunks loaded ahead (FP32 charges take twice the registers)
        uint32_t qw[TN / 32][QW];               // per 32-site chunk (a few live at a time)
        auto load_chunk = [&](const PairTile& tq, int c, uint32_t (&dst)[QW]) {
            const long b = (long)tq.n * 256 + (int)rank * PX_HN + lg * 32 + lane;
            const uint4* src =
                (const uint4*)((const uint8_t*)qt + (b * ld + 2 * tq.P * TC_M + c * 32) * QB);
            const bool in_row = c < TN / 64 || tq.slot1 >= 0;   // else past the end of the row
#pragma unroll
            for (int u = 0; u < QW / 4; ++u) {
                const uint4 v = in_row ? __ldg(src + u) : make_uint4(0u, 0u, 0u, 0u);
                dst[4 * u] = v.x;
                dst[4 * u + 1] = v.y;
                dst[4 * u + 2] = v.z;
                dst[4 * u + 3] = v.w;
            }
        };
        if (w0 < w1)
#pragma unroll
            for (int c = 0; c < PF; ++c) load_chunk(work[w0], c, qw[c]);
        int tl = 0;
        for (int wi = w0; wi < w1; ++wi, ++tl) {
            const PairTile tile = work[wi];
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            double s0 = 0.0, s1 = 0.0;              // panels 2P and 2P + 1
#pragma unroll
            for (int c = 0; c < TN / 32; ++c) {
                if (c + PF < TN / 32) load_chunk(tile, c + PF, qw[c + PF]);
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * TN) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                if (c == TN / 32 - 1) {
                    // the accumulator rows have been read: the MMA may start the tile after next in them
                    goacd::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0) goacd::mbar_arrive(&tempty[acc_i]);
                        else goacd::mbar_arrive_cluster(goacd::mapa_shared(goacd::smem_u32(&tempty[acc_i]), 0));
                    }
                }
                float a4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    // BF16 pairs widen to FP32 by position; FP32 charges are taken as they are
                    const float q0 = TF32 ? __uint_as_float(qw[c][j]) : __uint_as_float(qw[c][j / 2] << 16);
                    const float q1 = TF32 ? __uint_as_float(qw[c][j + 1]) : __uint_as_float(qw[c][j / 2] & 0xffff0000u);
                    a4[(j / 2) & 3] = fmaf(q0, __uint_as_float(r[j]), a4[(j / 2) & 3]);
                    a4[(j / 2) & 3] = fmaf(q1, __uint_as_float(r[j + 1]), a4[(j / 2) & 3]);
                }
                const double cs = (double)((a4[0] + a4[1]) + (a4[2] + a4[3]));
                if (c < TN / 64) s0 += cs;
                else s1 += cs;
            }
            if (wi + 1 < w1)
#pragma unroll
                for (int c = 0; c < PF; ++c) load_chunk(work[wi + 1], c, qw[c]);
            if (ok) {
                const long b = (long)tile.n * 256 + (int)rank * PX_HN + lg * 32 + lane;
                partial[(long)tile.slot0 * Bpad + b] = s0;
                if (tile.slot1 >= 0) partial[(long)tile.slot1 * Bpad + b] = s1;
            }
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::cluster_sync();                      // no CTA leaves while its peer may still reach its memory
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc_pair(tmem, 2 * TN);
    }
}

// Exact form with the configurations on the tensor-memory lanes: a tile is
// 128 configurations (M, rows of Q^T) x one pair-panel of 256 sites (N, the
// rows 256 P .. 256 P + 255 of digit t of J', i.e. panels 2P and 2P + 1) over
// the pair-panel's k-range (from 256 P; the host may cut it into chunks).  The
// accumulator row of configuration b then holds Phi_t,ib for the tile's 256
// sites, and the epilogue thread that owns the row forms
// P_t,I,b = sum_i q_bi Phi_t,ib over each panel's 128 sites by itself: no
// cross-lane reduction, no shared memory, no barrier between the epilogue
// warps.  The pair-panel's first two k-blocks meet panel 2P + 1 below its
// diagonal, where J' is zero: unless they are the whole tile they go last, as
// N = 128 MMAs over panel 2P's rows (loaded through a 128-row tensor map of
// J'); a pair-panel without panel 2P + 1 (odd panel count) runs N = 128 MMAs
// throughout.  The charges come from the int8 copy of Q^T (int16 when SPLIT)
// that k_make_qt writes beside the FP16 operand: 256 contiguous bytes (512)
// per configuration and tile, loaded before the tile's accumulator is ready.  Each 32-site chunk of
// products is summed in int32 under the same host bound as the one-CTA kernel
// (32 max|q a| < 2^31), the chunks in 64 bits; SPLIT sums the products in 64
// bits directly.  Work units and slots are pair_schedule's.
constexpr int CT_M = 128;                       // configurations per tile (TMEM lanes)
constexpr int CT_N = 256;                       // sites per tile (TMEM columns): one pair-panel
constexpr int CT_STAGE = A_TILE + B_TILE;       // 48 KB: 128 rows of Q^T, 256 rows of J'
constexpr int CT_STAGES = 4;
constexpr int CT_SMEM = CT_STAGES * CT_STAGE + 1024 + 256;

// The i-th k-block of a tile in processing order and whether its MMAs are
// N = 128: the range after the pair-panel's first two k-blocks first, those two
// (the head) last.
struct CtStep {
    int kb;
    bool narrow;
};
__device__ __forceinline__ CtStep ct_step(const PairTile& tile, int i)
{
    const int kp = 4 * tile.P;
    const bool single = tile.slot1 < 0;
    const int h1 = (tile.kb0 == kp && tile.kb1 > kp + 2) ? kp + 2 : tile.kb0;
    const int nrest = tile.kb1 - h1;
    const int kb = i < nrest ? h1 + i : tile.kb0 + (i - nrest);
    return CtStep{kb, single || kb < h1};
}

template <bool SPLIT>
__global__ void __launch_bounds__(192, SPLIT ? 1 : 2)
    k_score_exact_ct(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmJ,
                     const __grid_constant__ CUtensorMap tmJn, const PairTile* __restrict__ work,
                     const int* __restrict__ work_start, int ld, int T, const void* __restrict__ qi,
                     double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    static_assert(CT_STAGES * CT_STAGE + 1024 + 256 <= CT_SMEM, "stages exceed the dynamic shared memory");
    uint64_t* full = (uint64_t*)(smem + CT_STAGES * CT_STAGE);
    uint64_t* empty = full + CT_STAGES;
    uint64_t* tfull = empty + CT_STAGES;        // [2] accumulator ready
    uint64_t* tempty = tfull + 2;               // [2] accumulator drained
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w0 = work_start[blockIdx.x], w1 = work_start[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < CT_STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmQ);
        goacd::prefetch_tmap(&tmJ);
        goacd::prefetch_tmap(&tmJn);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, 2 * CT_N);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // launched as a dependent of k_make_qt: the set-up above overlaps its tail
    goacd::pdl_wait();
    goacd::pdl_trigger();

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int it = 0;
            for (int wi = w0; wi < w1 && !*abort_flag; ++wi) {
                const PairTile tile = work[wi];
                const int nsteps = tile.kb1 - tile.kb0;
                const int jrow = tile.t * ld + 2 * tile.P * TC_M;
                for (int i = 0; i < nsteps; ++i, ++it) {
                    const int s = it % CT_STAGES;
                    const uint32_t use = (uint32_t)(it / CT_STAGES);
                    if (it >= CT_STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    const CtStep k = ct_step(tile, i);
                    uint8_t* st = smem + s * CT_STAGE;
                    goacd::mbar_arrive_expect_tx(&full[s], A_TILE + (k.narrow ? A_TILE : B_TILE));
                    goacd::tma_load_2d(st, &tmQ, &full[s], k.kb * 64, tile.n * CT_M);
                    goacd::tma_load_2d(st + A_TILE, k.narrow ? &tmJn : &tmJ, &full[s], k.kb * 64, jrow);
                }
            }
            if (*abort_flag)
                for (int k = it - CT_STAGES < 0 ? 0 : it - CT_STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % CT_STAGES], (uint32_t)(k / CT_STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idw = goacd::idesc_f32acc(0u, CT_M, CT_N);    // FP16 charges and digits
            constexpr uint32_t idn = goacd::idesc_f32acc(0u, CT_M, CT_N / 2);
            int it = 0, tl = 0;
            for (int wi = w0; wi < w1; ++wi, ++tl) {
                const PairTile tile = work[wi];
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * CT_N);
                const int nsteps = tile.kb1 - tile.kb0;
                for (int i = 0; i < nsteps; ++i, ++it) {
                    if (*abort_flag) break;
                    const int s = it % CT_STAGES;
                    const uint32_t use = (uint32_t)(it / CT_STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t idesc = ct_step(tile, i).narrow ? idn : idw;
                    const uint32_t a0 = goacd::smem_u32(smem + s * CT_STAGE);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        goacd::mma_bf16(d_tmem, goacd::sdesc_k128(a0 + kk * 32),
                                        goacd::sdesc_k128(a0 + A_TILE + kk * 32), idesc,
                                        (i != 0 || kk != 0) ? 1u : 0u);
                    goacd::mma_commit(&empty[s]);
                }
                goacd::mma_commit(&tfull[acc_i]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5, one configuration per thread ----------------
        const int lg = warp & 3;
        constexpr int QPW = SPLIT ? 2 : 4;          // charges per 32-bit word
        uint32_t qp[CT_N / QPW];
        auto load_q = [&](const PairTile& tq) {
            const long b = (long)tq.n * CT_M + lg * 32 + lane;
            const uint4* src = (const uint4*)((const uint8_t*)qi + (b * ld + 2 * tq.P * TC_M) * (SPLIT ? 2 : 1));
            const bool two = tq.slot1 >= 0;     // else the sites past panel 2P lie outside the row
#pragma unroll
            for (int u = 0; u < CT_N / QPW / 4; ++u) {
                const uint4 v = (u < CT_N / QPW / 8 || two) ? __ldg(src + u) : make_uint4(0u, 0u, 0u, 0u);
                qp[4 * u] = v.x;
                qp[4 * u + 1] = v.y;
                qp[4 * u + 2] = v.z;
                qp[4 * u + 3] = v.w;
            }
        };
        if (w0 < w1) load_q(work[w0]);
        int tl = 0;
        for (int wi = w0; wi < w1; ++wi, ++tl) {
            const PairTile tile = work[wi];
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            long long s0 = 0, s1 = 0;               // panels 2P and 2P + 1
#pragma unroll
            for (int c = 0; c < CT_N / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * CT_N) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                if (c == CT_N / 32 - 1) {
                    // the accumulator has been read: the MMA warp may start the tile after next in it
                    goacd::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) goacd::mbar_arrive(&tempty[acc_i]);
                }
                long long cs;
                if constexpr (SPLIT) {
                    cs = 0;
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const uint32_t w = qp[(c * 32 + j) / 2];
                        cs += (long long)__float2int_rn(__uint_as_float(r[j])) * ct_charge<true, 0>(w);
                        cs += (long long)__float2int_rn(__uint_as_float(r[j + 1])) * ct_charge<true, 1>(w);
                    }
                } else {
                    int sum = 0;                    // |a| < 2^24 exact in FP32; 32 max|q a| < 2^31
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const uint32_t w = qp[(c * 32 + j) / 4];
                        sum += __float2int_rn(__uint_as_float(r[j])) * ct_charge<false, 0>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 1])) * ct_charge<false, 1>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 2])) * ct_charge<false, 2>(w);
                        sum += __float2int_rn(__uint_as_float(r[j + 3])) * ct_charge<false, 3>(w);
                    }
                    cs = sum;
                }
                if (c < CT_N / 64) s0 += cs;
                else s1 += cs;
            }
            if (wi + 1 < w1) load_q(work[wi + 1]);
            if (ok) {
                const long b = (long)tile.n * CT_M + lg * 32 + lane;
                partial[((long)tile.slot0 * T + tile.t) * Bpad + b] = (double)s0;
                if (tile.slot1 >= 0) partial[((long)tile.slot1 * T + tile.t) * Bpad + b] = (double)s1;
            }
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, 2 * CT_N);
    }
}

// Per 128-row panel I of the symmetric operand (sym != 0) or of J itself:
// e_I with max |J'| (max |J|) < 2^e_I.
__global__ void k_panel_exp(const double* __restrict__ J, int ld, int sym, int* __restrict__ pexp)
{
    __shared__ double red[256];
    const int I = blockIdx.x;
    double m = 0.0;
    for (long e = threadIdx.x; e < (long)TC_M * ld; e += blockDim.x) {
        const int r = (int)(e / ld), j = (int)(e % ld);
        const int i = I * TC_M + r;
        if (sym && j / TC_M < I) continue;
        const double v = fabs(J[(long)i * ld + j]) * (sym && j / TC_M > I ? 2.0 : 1.0);
        m = fmax(m, v);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        if (red[0] > 0.0) frexp(red[0], &e);     // red < 2^e
        pexp[I] = e;
    }
}

// FP16 hi / lo of J_vv 2^(15 - e_I) (e_I of row i's panel, max |J| < 2^e_I, so
// every scaled entry is below 2^15): out[0][i][j] = hi, out[1][i][j] = lo, each
// the FP16 rounding of what the parts before it leave.
__global__ void k_split_f16_full(const double* __restrict__ J, int ld, const int* __restrict__ pexp,
                                 __half* __restrict__ out)
{
    const long n = (long)ld * ld;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld);
        const double x = ldexp(J[e], 15 - pexp[i / TC_M]);
        const __half hi = __double2half(x);
        out[e] = hi;
        out[n + e] = __double2half(x - (double)__half2float(hi));
    }
}

// Digit t of J'/2^e_I (sym != 0) or J/2^e_I at [t][i][j]: a_t = rint of the
// remainder scaled by 2^(r-1+rt), stored in FP16 (|a_t| <= 2^(r-1) <= 1024).
__global__ void k_split_digits(const double* __restrict__ J, int ld, int sym, const int* __restrict__ pexp, int r,
                               int T, __half* __restrict__ out)
{
    const long n = (long)ld * ld;
    const double radix = ldexp(1.0, r);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld), j = (int)(e % ld);
        const int bi = i / TC_M, bj = j / TC_M;
        double x = !sym ? J[e] : (bj < bi ? 0.0 : (bj > bi ? 2.0 * J[e] : J[e]));
        x = ldexp(x, r - 1 - pexp[bi]);           // |x| < 2^(r-1)
        for (int t = 0; t < T; ++t) {
            const double a = rint(x);
            out[t * n + e] = __double2half((double)a);
            x = (x - a) * radix;
        }
    }
}

// Potentials Phi = J_vv Q through the integer-digit split of J_vv itself (the
// exact-form counterpart of the FP64 GEMM, used to start FP64 chains).  Tile =
// (panel I, 256 configurations, digit t) over the whole k-range; all tiles
// have the same length and are dealt round-robin to the persistent grid, digit
// fastest so that concurrent CTAs share Q tiles in L2.  Same stages, MMA shape
// and double-buffered TMEM accumulators as k_score_exact; the epilogue stores
// each exact digit sum as a 32-bit integer, Phi_t[b][v].
__global__ void __launch_bounds__(192, 1)
    k_phi_exact(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int ntiles,
                int nbm, int nkb, int ld, int Bpad, int T, int* __restrict__ Phi, int* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + EX_STAGES * EX_STAGE);
    uint64_t* empty = full + EX_STAGES;
    uint64_t* tfull = empty + EX_STAGES;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < EX_STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            goacd::mbar_init(&tfull[a], 1);
            goacd::mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, 2 * TC_N);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int id = blockIdx.x; id < ntiles && !*abort_flag; id += gridDim.x) {
                const int t = id % T, I = (id / T) % nbm, n = id / (T * nbm);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % EX_STAGES;
                    const uint32_t use = (uint32_t)(it / EX_STAGES);
                    if (it >= EX_STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, it);
                        break;
                    }
                    if (*abort_flag) break;
                    uint8_t* st = smem + s * EX_STAGE;
                    goacd::mbar_arrive_expect_tx(&full[s], EX_STAGE);
                    goacd::tma_load_2d(st, &tmA, &full[s], kb * 64, t * ld + I * TC_M);
                    goacd::tma_load_2d(st + A_TILE, &tmB, &full[s], kb * 64, n * TC_N);
                }
            }
            if (*abort_flag)
                for (int k = it - EX_STAGES < 0 ? 0 : it - EX_STAGES; k < it; ++k)
                    if (!goacd::mbar_wait_bounded(&full[k % EX_STAGES], (uint32_t)(k / EX_STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, k);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(0u, TC_M, TC_N);   // FP16 digits and charges
            int it = 0, tl = 0;
            for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++tl) {
                const int acc_i = tl & 1;
                const uint32_t ause = (uint32_t)(tl >> 1);
                if (tl >= 2 && !goacd::mbar_wait_bounded(&tempty[acc_i], (ause - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, -1 - tl);
                }
                goacd::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * TC_N);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    if (*abort_flag) break;
                    const int s = it % EX_STAGES;
                    const uint32_t use = (uint32_t)(it / EX_STAGES);
                    if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                        *abort_flag = 1;
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, it);
                        break;
                    }
                    goacd::tc_fence_after();
                    const uint32_t a0 = goacd::smem_u32(smem + s * EX_STAGE);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        goacd::mma_bf16(d_tmem, goacd::sdesc_k128(a0 + kk * 32),
                                        goacd::sdesc_k128(a0 + A_TILE + kk * 32), idesc,
                                        (kb != 0 || kk != 0) ? 1u : 0u);
                    goacd::mma_commit(&empty[s]);
                }
                goacd::mma_commit(&tfull[acc_i]);
            }
        }
        __syncwarp();
    } else {
        const int lg = warp & 3;
        int tl = 0;
        for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++tl) {
            const int t = id % T, I = (id / T) % nbm, n = id / (T * nbm);
            const int acc_i = tl & 1;
            const uint32_t ause = (uint32_t)(tl >> 1);
            const bool ok = goacd::mbar_wait_bounded(&tfull[acc_i], ause & 1, WAIT_LIMIT) && !*abort_flag;
            if (!ok && lane == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, tl);
            goacd::tc_fence_after();
            const int v = I * TC_M + lg * 32 + lane;
            int* dst = Phi + ((long)t * Bpad + (long)n * TC_N) * ld + v;
#pragma unroll 1
            for (int c = 0; c < TC_N / 32; ++c) {
                uint32_t r[32];
                goacd::tmem_ld_32x32b_x32(tmem + (uint32_t)(acc_i * TC_N) + ((uint32_t)(lg * 32) << 16) +
                                              (uint32_t)(c * 32),
                                          r);
                goacd::tmem_ld_wait();
                if (ok)
#pragma unroll
                    for (int j = 0; j < 32; ++j) dst[(long)(c * 32 + j) * ld] = __float2int_rn(__uint_as_float(r[j]));
            }
            goacd::tc_fence_before();
            __syncwarp();
            if (lane == 0) goacd::mbar_arrive(&tempty[acc_i]);
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, 2 * TC_N);
    }
}

// phi_bv = 2^(e_I - (r-1) - kq) sum_t 2^-rt Phi_t[b][v] + phi_fix_v (digits
// smallest first) and E_b = sum_v q_bv (phi_bv + phi_fix_v) + E_const, one block
// per configuration, fixed reduction order.
template <typename PT>
__global__ void __launch_bounds__(256)
    k_phi_exact_finish(const int* __restrict__ Phi, int Bpad, int ld, int Nv, const int* __restrict__ pexp, int kq,
                       int r, int T, const double* __restrict__ phifix, const int8_t* __restrict__ species,
                       const double* __restrict__ z, double E_const, PT* __restrict__ phi_out,
                       double* __restrict__ E_out)
{
    __shared__ double red[256];
    const int b = blockIdx.x;
    double e = 0.0;
    for (int v = threadIdx.x; v < Nv; v += blockDim.x) {
        double d = 0.0;
        for (int t = T - 1; t >= 0; --t) d += (double)Phi[((long)t * Bpad + b) * ld + v] * pow2(-r * t);
        const double pf = phifix[v];
        const double ph = d * pow2(pexp[v / TC_M] - (r - 1) - kq) + pf;
        if (phi_out) phi_out[(long)b * Nv + v] = (PT)ph;      // FP32 chains: phi rounded once
        e += z[species[(long)b * Nv + v]] * (ph + pf);
    }
    if (!E_out) return;
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) E_out[b] = red[0] + E_const;
}

// Symmetric operand: J'_ij = J_ij on diagonal 128-blocks, 2 J_ij above them,
// 0 below, so that q^T J q = sum over the upper block triangle of q_I^T J'_IJ q_J.
__device__ __forceinline__ double sym_upper(const double* J, long e, int ld)
{
    const int i = (int)(e / ld), j = (int)(e % ld);
    const int bi = i / 128, bj = j / 128;
    return bj < bi ? 0.0 : (bj > bi ? 2.0 * J[e] : J[e]);
}

__global__ void k_split_bf16(const double* __restrict__ J, long n, int ld, __nv_bfloat16* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double x = sym_upper(J, e, ld);
        const __nv_bfloat16 t1 = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(t1);
        const __nv_bfloat16 t2 = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(t2);
        const __nv_bfloat16 t3 = __double2bfloat16(r2);
        out[e] = t1;
        out[n + e] = t2;
        out[2 * n + e] = t3;
    }
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void k_split_tf32(const double* __restrict__ J, long n, int ld, float* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double x = sym_upper(J, e, ld);
        const float hi = to_tf32((float)x);
        const float lo = to_tf32((float)(x - (double)hi));
        out[e] = hi;
        out[n + e] = lo;
    }
}

__global__ void k_copy_f32(const double* __restrict__ J, long n, float* __restrict__ out,
                           const double* __restrict__ diag, int Nv, float* __restrict__ diag_out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        out[e] = (float)J[e];
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < Nv; e += (long)gridDim.x * blockDim.x)
        diag_out[e] = (float)diag[e];
}

// Q^T[b][v] = z[species[b][v]] in BF16, FP16 or FP32, zero padded to Bpad x ld, one
// block of 128 threads per configuration row; a thread converts two chunks of
// 16 species per step (one 16-byte load each when the row is 16-byte aligned,
// both issued before either is converted), 16-byte stores.  With fixed ions
// also lin[b] = sum_v q_bv 2 phi_fix_v in FP64 (fixed reduction order).  FP16
// with qbytes 1 or 2: the same integer charges also as int8 or int16 at
// qi[b][v] (the exact form's epilogue operand).
constexpr int MQ_T = 128;

template <typename QT>
__device__ __forceinline__ void make_qt_chunk(const int8_t (&s16)[16], const float* zs, const double* __restrict__ z,
                                              const double* __restrict__ phifix, int v0, QT* __restrict__ row,
                                              double& acc, uint8_t* __restrict__ qrow, int qbytes)
{
    float q[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        q[u] = s16[u] >= 0 ? zs[s16[u]] : 0.0f;
        if (phifix && s16[u] >= 0) acc += z[s16[u]] * (2.0 * phifix[v0 + u]);
    }
    if constexpr (std::is_same<QT, __half>::value) {
        __align__(16) __half o[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) o[u] = __float2half_rn(q[u]);
        ((int4*)(row + v0))[0] = ((const int4*)o)[0];
        ((int4*)(row + v0))[1] = ((const int4*)o)[1];
        if (qbytes == 1) {
            // integer charges (the exact form's q are integers below 2^6 here)
            __align__(16) int8_t c[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) c[u] = (int8_t)__float2int_rn(q[u]);
            *(int4*)(qrow + v0) = *(const int4*)c;
        } else if (qbytes == 2) {
            __align__(16) int16_t c[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) c[u] = (int16_t)__float2int_rn(q[u]);
            ((int4*)(qrow + 2 * v0))[0] = ((const int4*)c)[0];
            ((int4*)(qrow + 2 * v0))[1] = ((const int4*)c)[1];
        }
    } else if constexpr (sizeof(QT) == 2) {
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) o[u] = __float2bfloat16(q[u]);
        ((int4*)(row + v0))[0] = ((const int4*)o)[0];
        ((int4*)(row + v0))[1] = ((const int4*)o)[1];
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) ((float4*)(row + v0))[u] = make_float4(q[4 * u], q[4 * u + 1], q[4 * u + 2], q[4 * u + 3]);
    }
}

__device__ __forceinline__ void make_qt_load(const int8_t* __restrict__ src, int b, int B, int Nv, bool aligned, int v0,
                                             int8_t (&s16)[16])
{
    if (b < B && aligned && v0 + 16 <= Nv) {
        *(int4*)s16 = *(const int4*)(src + v0);
    } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) s16[u] = (b < B && v0 + u < Nv) ? src[v0 + u] : (int8_t)-1;
    }
}

template <typename QT>
__global__ void __launch_bounds__(MQ_T) k_make_qt(const int8_t* __restrict__ species, int B, int Nv,
                                                  const double* __restrict__ zq, const double* __restrict__ z, int ld,
                                                  QT* __restrict__ qt, const double* __restrict__ phifix,
                                                  double* __restrict__ lin, void* __restrict__ qi, int qbytes)
{
    __shared__ float zs[64];
    __shared__ double red[MQ_T];
    goacd::pdl_trigger();       // the scoring kernel may set itself up meanwhile
    if (threadIdx.x < 64) zs[threadIdx.x] = (float)zq[threadIdx.x];
    __syncthreads();
    const int b = blockIdx.x;
    QT* row = qt + (long)b * ld;
    const int8_t* src = species + (long)b * Nv;
    const bool aligned = ((Nv & 15) == 0) && (((uintptr_t)species & 15) == 0);
    uint8_t* qrow = qi ? (uint8_t*)qi + (long)b * ld * qbytes : nullptr;
    if (!qi) qbytes = 0;
    double acc = 0.0;
    for (int v0 = threadIdx.x * 16; v0 < ld; v0 += 2 * MQ_T * 16) {   // ld is a multiple of 128
        const int v1 = v0 + MQ_T * 16;
        int8_t sa[16], sb[16];
        make_qt_load(src, b, B, Nv, aligned, v0, sa);
        if (v1 < ld) make_qt_load(src, b, B, Nv, aligned, v1, sb);
        make_qt_chunk<QT>(sa, zs, z, phifix, v0, row, acc, qrow, qbytes);
        if (v1 < ld) make_qt_chunk<QT>(sb, zs, z, phifix, v1, row, acc, qrow, qbytes);
    }
    if (phifix == nullptr || b >= B) return;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = MQ_T / 2; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lin[b] = red[0];
}

constexpr int EX_TMAX = 6;                     // most digits of the exact form

// E_b = 2^-2kq sum_I 2^(e_I - (r-1)) sum_t 2^-rt P_t,I,b + lin_b + E_const,
// P_t,I,b the sum of panel I's k-chunk partials (slots pslot[I] ..
// pslot[I+1]) of digit t: exact integers below 2^53, so the result does not
// depend on how the panel's k-range was split.  One block of 32 warps per 32
// configurations: lane = configuration (coalesced loads of the partials), warp
// w takes panels w, w + 32, ... (up to Nv = 4,096 one panel per warp: one round
// trip for the panel's slot bounds and one for its partials); a panel's T
// partials are loaded together, the digits added smallest first and the 32
// warp sums in a fixed order (deterministic); the scalings are exact powers of
// two.
constexpr int FX_WARPS = 32;
__global__ void __launch_bounds__(FX_WARPS * 32)
    k_finish_exact(const double* __restrict__ partial, int npanels, const int* __restrict__ pslot,
                   const int* __restrict__ pexp, int Bpad, int B, int r, int T, int kq2, double E_const,
                   const double* __restrict__ lin, double* __restrict__ E)
{
    __shared__ double red[FX_WARPS][33];
    goacd::pdl_wait();          // the digit sums of the scoring kernel
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (b < B)
        for (int m = warp; m < npanels; m += FX_WARPS) {
            const int s0 = pslot[m], s1 = pslot[m + 1];
            double P[EX_TMAX];
#pragma unroll
            for (int t = 0; t < EX_TMAX; ++t) P[t] = 0.0;
            for (int sl = s0; sl < s1; ++sl) {
                const double* ps = partial + (long)sl * T * Bpad + b;
#pragma unroll
                for (int t = 0; t < EX_TMAX; ++t)
                    if (t < T) P[t] += ps[(long)t * Bpad];
            }
            double d = 0.0;
#pragma unroll
            for (int t = EX_TMAX - 1; t >= 0; --t)
                if (t < T) d += P[t] * pow2(-r * t);
            s += d * pow2(pexp[m] - (r - 1));
        }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && b < B) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < FX_WARPS; ++w) tot += red[w][lane];
        E[b] = tot * pow2(-kq2) + (lin ? lin[b] : 0.0) + E_const;
    }
}

// E_b = sum over the partial-sum slots in order + lin_b + E_const.
__global__ void k_finish_tc(const double* __restrict__ partial, int nslots, int Bpad, int B, double E_const,
                            const double* __restrict__ lin, double* __restrict__ E)
{
    goacd::pdl_wait();          // the partial sums of the scoring kernel
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
    for (int m = 0; m < nslots; ++m) s += partial[(long)m * Bpad + b];
    E[b] = s + (lin ? lin[b] : 0.0) + E_const;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Opt a kernel into its large dynamic shared memory on the given (current)
// device, once per device: the attribute belongs to the device, so a process
// with contexts on several GPUs must set it on each.
goac_status smem_attr_once(const void* kern, int smem, std::atomic<uint64_t>& done, int device)
{
    const uint64_t bit = 1ull << (device & 63);
    if (done.load() & bit) return GOAC_OK;
    GOAC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done.fetch_or(bit);
    return GOAC_OK;
}

// 2D K-major tensor map: inner dim = `inner` elements (row pitch `pitch_elems`),
// outer dim = `rows`; box = 128 bytes x box_rows, 128-byte swizzle.
goac_status make_map(CUtensorMap* map, void* base, CUtensorMapDataType dt, int elem_bytes, long inner, long rows,
                     long pitch_elems, int box_rows, int row_bytes = ROW_BYTES)
{
    auto enc = get_encode();
    if (!enc) return goac::fail(GOAC_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    if (((uintptr_t)base & 15) != 0 || (pitch_elems * elem_bytes) % 16 != 0)
        return goac::fail(GOAC_ERR_INTERNAL, "tensor map base / pitch not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * elem_bytes)};
    if (row_bytes != 128 && row_bytes != 64) return goac::fail(GOAC_ERR_INTERNAL, "tensor map row bytes");
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return goac::fail(GOAC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return GOAC_OK;
}

// Number of tiles (x) and partial-sum slots (y) of a shape: panel I has
// nbm - I blocks of 128 columns, cut into chunks of kc blocks (kc = 0: one).
int2 tc_tile_count(int nbm, int nbn, int T, int kc)
{
    long tiles = 0;
    int slots = 0;
    for (int I = 0; I < nbm; ++I) {
        const int nch = kc > 0 ? (nbm - I + kc - 1) / kc : 1;
        slots += nch;
        tiles += (long)nch * nbn * T;
    }
    return make_int2((int)std::min<long>(tiles, 1L << 30), slots);
}

// Longest-processing-time schedule of the tiles (panel I, configuration tile
// n, k-chunk, digit t) over the CTAs of a persistent grid, cached per problem
// for the last shape.  Panel I's k-range (k-blocks from I kbm to nkb, kbm
// k-blocks per 128 columns) is cut into chunks of kc 128-column blocks (kc = 0:
// one chunk); each (I, chunk) is one partial-sum slot, slots numbered panel by
// panel, so the slots of panel I are pslot[I] .. pslot[I+1].  Tiles go
// longest first to the least-loaded CTA (ties: the lowest index); each CTA
// then runs its tiles longest, shortest, second longest, ... so that the
// epilogue of a short tile (which can take longer than its MMAs) overlaps the
// MMAs of a long one through the two TMEM accumulators.
goac_status tc_schedule(TcSched& sc, cudaStream_t stream, int nbm, int nbn, int T, int kc, int kbm, int grid,
                        const TcTile** work,
                        const int** starts, const int** pslot)
{
    if (nbm <= 0 || nbm >= (1 << 18) || nbn <= 0 || nbn >= (1 << 26) || grid <= 0 || grid >= (1 << 20) || T < 1 ||
        T > 15 || kc < 0 || kc >= (1 << 16) || kbm < 1 || kbm > 15)
        return goac::fail(GOAC_ERR_INVALID_ARG, "tile schedule: shape out of range");
    const uint64_t k0 = ((uint64_t)nbm << 46) | ((uint64_t)nbn << 20) | (uint64_t)grid;
    const uint64_t k1 = ((uint64_t)T << 24) | ((uint64_t)kc << 8) | (uint64_t)kbm;
    if (sc.key[0] != k0 || sc.key[1] != k1) {
        const int nkb = nbm * kbm;
        std::vector<TcTile> tiles;
        std::vector<int> ps(nbm + 1, 0);
        int slot = 0;
        for (int I = 0; I < nbm; ++I) {
            ps[I] = slot;
            const int step = kc > 0 ? kc * kbm : nkb - I * kbm;
            for (int kb0 = I * kbm; kb0 < nkb; kb0 += step, ++slot) {
                const int kb1 = std::min(nkb, kb0 + step);
                for (int n = 0; n < nbn; ++n)
                    for (int t = 0; t < T; ++t) tiles.push_back(TcTile{I, n, kb0, kb1, slot, t});
            }
        }
        ps[nbm] = slot;
        std::stable_sort(tiles.begin(), tiles.end(),
                         [](const TcTile& a, const TcTile& b) { return a.kb1 - a.kb0 > b.kb1 - b.kb0; });
        // each tile goes to the least-loaded CTA (ties: the lowest index), a min-heap on (load, CTA)
        std::vector<std::vector<TcTile>> per(grid);
        std::priority_queue<std::pair<long, int>, std::vector<std::pair<long, int>>,
                            std::greater<std::pair<long, int>>>
            heap;
        for (int c = 0; c < grid; ++c) heap.push({0L, c});
        for (const TcTile& t : tiles) {
            const auto [ld0, best] = heap.top();
            heap.pop();
            per[best].push_back(t);
            heap.push({ld0 + (t.kb1 - t.kb0) / kbm + 1, best});   // 128-column blocks, +1 for the epilogue
        }
        std::vector<TcTile> flat;
        std::vector<int> st(grid + 1, 0);
        for (int c = 0; c < grid; ++c) {
            st[c] = (int)flat.size();
            // longest, shortest, second longest, ...: a short tile's epilogue overlaps a long tile's MMAs
            for (int lo = 0, hi = (int)per[c].size() - 1; lo <= hi; ++lo, --hi) {
                flat.push_back(per[c][lo]);
                if (hi > lo) flat.push_back(per[c][hi]);
            }
        }
        st[grid] = (int)flat.size();
        const size_t bytes = sizeof(TcTile) * flat.size() + sizeof(int) * (grid + 1 + nbm + 1) + 64;
        goac_status rc = goac::ensure(sc.buf, bytes);
        if (rc) return rc;
        TcTile* dw = (TcTile*)sc.buf.ptr;
        int* ds = (int*)(dw + flat.size());
        // stream-ordered: a launch still reading the previous schedule finishes first
        GOAC_CUDA(cudaMemcpyAsync(dw, flat.data(), sizeof(TcTile) * flat.size(), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaMemcpyAsync(ds, st.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaMemcpyAsync(ds + grid + 1, ps.data(), sizeof(int) * (nbm + 1), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaStreamSynchronize(stream));   // the host vectors go out of scope
        sc.key[0] = k0;
        sc.key[1] = k1;
        sc.ntiles = (int)flat.size();
        sc.nslots = slot;
        sc.grid = grid;
    }
    *work = (const TcTile*)sc.buf.ptr;
    *starts = (const int*)((const TcTile*)sc.buf.ptr + sc.ntiles);
    if (pslot) *pslot = *starts + sc.grid + 1;
    return GOAC_OK;
}

template <int T, bool TF32, int TN>
goac_status launch_tc(goac_problem* p, const CUtensorMap& ma, const CUtensorMap& mb, int Bpad, int B, int kc,
                      const void* qt, double* part)
{
    using Cfg = TcCfg<T, TN>;
    auto kern = k_score_tc<T, TF32, TN>;
    static std::atomic<uint64_t> attr_done{0};
    {
        goac_status rc0 = smem_attr_once((const void*)kern, Cfg::SMEM, attr_done, p->ctx->device);
        if (rc0) return rc0;
    }
    const int ld = p->Nv_pad;
    const int nbm = ld / TC_M, nbn = (B + TN - 1) / TN;
    const int2 cnt = tc_tile_count(nbm, nbn, 1, kc);
    const int grid = std::min(cnt.x, p->ctx->num_sms);
    const TcTile* work = nullptr;
    const int* starts = nullptr;
    goac_status rc = tc_schedule(p->sched, p->ctx->stream, nbm, nbn, 1, kc, TF32 ? 4 : 2, grid, &work, &starts, nullptr);
    if (rc) return rc;
    goac::KTimer kt(p->ctx, goac::KID_SCORE_TC, p->ctx->stream);
    goac::launch_pdl(kern, grid, 192, Cfg::SMEM, p->ctx->stream, ma, mb, work, starts, ld, qt, ld, part, Bpad,
                     p->ctx->d_err);
    GOAC_LAUNCH_CHECK("k_score_tc");
    return GOAC_OK;
}

template <int TN, bool SPLIT>
goac_status launch_exact(goac_problem* p, const CUtensorMap& ma, const CUtensorMap& mb, int Bpad, int B, int kc,
                         double* part, const double* lin, double* E_out)
{
    using Cfg = ExCfg<TN>;
    auto kern = k_score_exact<TN, SPLIT>;
    static std::atomic<uint64_t> attr_done{0};
    goac_status rc = smem_attr_once((const void*)kern, Cfg::SMEM, attr_done, p->ctx->device);
    if (rc) return rc;
    const int ld = p->Nv_pad, T = p->dig_T;
    const int nbm = ld / TC_M, nbn = (B + TN - 1) / TN;
    const int2 cnt = tc_tile_count(nbm, nbn, T, kc);
    const int grid = std::min(cnt.x, p->ctx->num_sms);
    const TcTile* work = nullptr;
    const int* starts = nullptr;
    const int* pslot = nullptr;
    rc = tc_schedule(p->sched_ex, p->ctx->stream, nbm, nbn, T, kc, 2, grid, &work, &starts, &pslot);
    if (rc) return rc;
    {
        goac::KTimer kt(p->ctx, goac::KID_SCORE_TC, p->ctx->stream);
        goac::launch_pdl(kern, grid, 192, Cfg::SMEM, p->ctx->stream, ma, mb, work, starts, ld, T,
                         (const __half*)p->qt.ptr, part, Bpad, p->ctx->d_err);
        GOAC_LAUNCH_CHECK("k_score_exact");
    }
    goac::launch_pdl(k_finish_exact, (B + 31) / 32, FX_WARPS * 32, 0, p->ctx->stream, (const double*)part, nbm, pslot,
                     (const int*)p->dig_exp, Bpad, B, p->dig_r, T, 2 * p->dig_kq, p->E_const, lin, E_out);
    GOAC_LAUNCH_CHECK("k_finish_exact");
    return GOAC_OK;
}

// Schedule of the CTA-pair kernel: pair tiles (pair-panel P, configuration
// tile n, k-chunk, digit t) longest first over the pairs; panel I's k-chunk
// slots are numbered panel by panel (pslot[I] .. pslot[I+1]) as for the
// one-CTA kernel, with panel 2P + 1 chunked like its pair-panel.
goac_status pair_schedule(TcSched& sc, cudaStream_t stream, int nbm, int nbn, int T, int kc, int kbm, int npairs,
                          const PairTile** work, const int** starts, const int** pslot)
{
    if (nbm <= 0 || nbm >= (1 << 18) || nbn <= 0 || nbn >= (1 << 26) || npairs <= 0 || npairs >= (1 << 19) ||
        T < 1 || T > 15 || kc < 0 || kc >= (1 << 16) || kbm < 1 || kbm > 15)
        return goac::fail(GOAC_ERR_INVALID_ARG, "pair schedule: shape out of range");
    const uint64_t k0 = ((uint64_t)nbm << 46) | ((uint64_t)nbn << 20) | (uint64_t)npairs;
    const uint64_t k1 = (1ull << 40) | ((uint64_t)T << 24) | ((uint64_t)kc << 8) | (uint64_t)kbm;
    if (sc.key[0] != k0 || sc.key[1] != k1) {
        const int nkb = nbm * kbm, npp = (nbm + 1) / 2;
        std::vector<int> ps(nbm + 1, 0), nch(npp, 0);
        for (int P = 0; P < npp; ++P) {
            const int span = nkb - 2 * P * kbm;
            const int step = kc > 0 ? kc * kbm : span;
            nch[P] = (span + step - 1) / step;
        }
        int slot = 0;
        for (int I = 0; I < nbm; ++I) {
            ps[I] = slot;
            slot += nch[I / 2];
        }
        ps[nbm] = slot;
        std::vector<PairTile> tiles;
        for (int P = 0; P < npp; ++P) {
            const int step = kc > 0 ? kc * kbm : nkb - 2 * P * kbm;
            int c = 0;
            for (int kb0 = 2 * P * kbm; kb0 < nkb; kb0 += step, ++c) {
                const int kb1 = std::min(nkb, kb0 + step);
                const int s0 = ps[2 * P] + c, s1 = 2 * P + 1 < nbm ? ps[2 * P + 1] + c : -1;
                for (int n = 0; n < nbn; ++n)
                    for (int t = 0; t < T; ++t) tiles.push_back(PairTile{P, n, kb0, kb1, s0, s1, t});
            }
        }
        std::stable_sort(tiles.begin(), tiles.end(),
                         [](const PairTile& a, const PairTile& b) { return a.kb1 - a.kb0 > b.kb1 - b.kb0; });
        std::vector<std::vector<PairTile>> per(npairs);
        std::priority_queue<std::pair<long, int>, std::vector<std::pair<long, int>>,
                            std::greater<std::pair<long, int>>>
            heap;
        for (int c = 0; c < npairs; ++c) heap.push({0L, c});
        for (const PairTile& t : tiles) {
            const auto [ld0, best] = heap.top();
            heap.pop();
            per[best].push_back(t);
            heap.push({ld0 + (t.kb1 - t.kb0) / kbm + 1, best});
        }
        std::vector<PairTile> flat;
        std::vector<int> st(npairs + 1, 0);
        for (int c = 0; c < npairs; ++c) {
            st[c] = (int)flat.size();
            for (int lo = 0, hi = (int)per[c].size() - 1; lo <= hi; ++lo, --hi) {
                flat.push_back(per[c][lo]);
                if (hi > lo) flat.push_back(per[c][hi]);
            }
        }
        st[npairs] = (int)flat.size();
        const size_t bytes = sizeof(PairTile) * flat.size() + sizeof(int) * (npairs + 1 + nbm + 1) + 64;
        goac_status rc = goac::ensure(sc.buf, bytes);
        if (rc) return rc;
        PairTile* dw = (PairTile*)sc.buf.ptr;
        int* ds = (int*)(dw + flat.size());
        // stream-ordered: a launch still reading the previous schedule finishes first
        GOAC_CUDA(cudaMemcpyAsync(dw, flat.data(), sizeof(PairTile) * flat.size(), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaMemcpyAsync(ds, st.data(), sizeof(int) * (npairs + 1), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaMemcpyAsync(ds + npairs + 1, ps.data(), sizeof(int) * (nbm + 1), cudaMemcpyHostToDevice, stream));
        GOAC_CUDA(cudaStreamSynchronize(stream));   // the host vectors go out of scope
        sc.key[0] = k0;
        sc.key[1] = k1;
        sc.ntiles = (int)flat.size();
        sc.nslots = slot;
        sc.grid = npairs;
    }
    *work = (const PairTile*)sc.buf.ptr;
    *starts = (const int*)((const PairTile*)sc.buf.ptr + sc.ntiles);
    *pslot = *starts + sc.grid + 1;
    return GOAC_OK;
}

// Partial-sum slots of the pair kernel's shape (see pair_schedule).
int pair_slot_count(int nbm, int kc)
{
    int slot = 0;
    for (int I = 0; I < nbm; ++I) {
        const int span = 2 * nbm - 2 * 2 * (I / 2);
        const int step = kc > 0 ? kc * 2 : span;
        slot += (span + step - 1) / step;
    }
    return slot;
}

// CTA pairs that can be resident at once (clusters of two with the pair kernel's shared memory).
static int max_pairs(goac_problem* p)
{
    static std::atomic<int> cached[64] = {};
    const int dev = p->ctx->device & 63;
    int v = cached[dev].load();
    if (v > 0) return v;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (p->ctx->num_sms / 2));
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = PX_SMEM;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_score_exact_pair<true>, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = p->ctx->num_sms / 2;
    }
    n = std::min(n, p->ctx->num_sms / 2);
    cached[dev].store(n);
    return n;
}

template <bool SPLIT>
goac_status launch_exact_pair(goac_problem* p, const CUtensorMap& ma, const CUtensorMap& mb, int Bpad, int B, int kc,
                              double* part, const double* lin, double* E_out)
{
    static std::atomic<uint64_t> attr_done{0};
    goac_status rc = smem_attr_once((const void*)k_score_exact_pair<SPLIT>, PX_SMEM, attr_done, p->ctx->device);
    if (rc) return rc;
    const int ld = p->Nv_pad, T = p->dig_T;
    const int nbm = ld / TC_M, nbn = (B + 255) / 256, npp = (nbm + 1) / 2;
    long ntiles = 0;
    for (int P = 0; P < npp; ++P) {
        const int span = 2 * nbm - 4 * P;
        ntiles += (long)(kc > 0 ? (span + 2 * kc - 1) / (2 * kc) : 1) * nbn * T;
    }
    const int npairs = (int)std::min<long>(ntiles, max_pairs(p));
    const PairTile* work = nullptr;
    const int* starts = nullptr;
    const int* pslot = nullptr;
    rc = pair_schedule(p->sched_ex, p->ctx->stream, nbm, nbn, T, kc, 2, npairs, &work, &starts, &pslot);
    if (rc) return rc;
    {
        goac::KTimer kt(p->ctx, goac::KID_SCORE_TC, p->ctx->stream);
        goac::launch_pdl(k_score_exact_pair<SPLIT>, 2 * npairs, 192, PX_SMEM, p->ctx->stream, ma, mb, work, starts, ld, T,
                         (const void*)p->qi.ptr, part, Bpad, p->ctx->d_err);
        GOAC_LAUNCH_CHECK("k_score_exact_pair");
    }
    goac::launch_pdl(k_finish_exact, (B + 31) / 32, FX_WARPS * 32, 0, p->ctx->stream, (const double*)part, nbm, pslot,
                     (const int*)p->dig_exp, Bpad, B, p->dig_r, T, 2 * p->dig_kq, p->E_const, lin, E_out);
    GOAC_LAUNCH_CHECK("k_finish_exact");
    return GOAC_OK;
}

// The configuration-lane kernel: pair_schedule's work units over a persistent
// grid of one CTA per SM (128-configuration blocks), then k_finish_exact.
template <bool SPLIT>
goac_status launch_exact_ct(goac_problem* p, const CUtensorMap& mq, const CUtensorMap& mj, const CUtensorMap& mjn,
                            int Bpad, int B, int kc, double* part, const double* lin, double* E_out)
{
    static std::atomic<uint64_t> attr_done{0};
    goac_status rc = smem_attr_once((const void*)k_score_exact_ct<SPLIT>, CT_SMEM, attr_done, p->ctx->device);
    if (rc) return rc;
    const int ld = p->Nv_pad, T = p->dig_T;
    const int nbm = ld / TC_M, nbn = (B + CT_M - 1) / CT_M, npp = (nbm + 1) / 2;
    long ntiles = 0;
    for (int P = 0; P < npp; ++P) {
        const int span = 2 * nbm - 4 * P;
        ntiles += (long)(kc > 0 ? (span + 2 * kc - 1) / (2 * kc) : 1) * nbn * T;
    }
    const int grid = (int)std::min<long>(ntiles, p->ctx->num_sms);
    const PairTile* work = nullptr;
    const int* starts = nullptr;
    const int* pslot = nullptr;
    rc = pair_schedule(p->sched_ex, p->ctx->stream, nbm, nbn, T, kc, 2, grid, &work, &starts, &pslot);
    if (rc) return rc;
    {
        goac::KTimer kt(p->ctx, goac::KID_SCORE_TC, p->ctx->stream);
        goac::launch_pdl(k_score_exact_ct<SPLIT>, grid, 192, CT_SMEM, p->ctx->stream, mq, mj, mjn, work, starts, ld,
                         T, (const void*)p->qi.ptr, part, Bpad, p->ctx->d_err);
        GOAC_LAUNCH_CHECK("k_score_exact_ct");
    }
    goac::launch_pdl(k_finish_exact, (B + 31) / 32, FX_WARPS * 32, 0, p->ctx->stream, (const double*)part, nbm, pslot,
                     (const int*)p->dig_exp, Bpad, B, p->dig_r, T, 2 * p->dig_kq, p->E_const, lin, E_out);
    GOAC_LAUNCH_CHECK("k_finish_exact");
    return GOAC_OK;
}

// The split forms' CTA-pair kernel: pair_schedule's work units (one digit
// index; 2 k-blocks per 128 columns in BF16, 4 in TF32) over the resident
// clusters, then k_finish_tc.
template <int T, bool TF32>
goac_status launch_tc_pair(goac_problem* p, const CUtensorMap& mq, const CUtensorMap& mj, int Bpad, int B, int kc,
                           double* part)
{
    using Cfg = TpCfg<T>;
    static_assert(Cfg::SMEM <= PX_SMEM, "the resident-pair count is taken with the exact pair kernel's memory");
    static std::atomic<uint64_t> attr_done{0};
    goac_status rc = smem_attr_once((const void*)k_score_tc_pair<T, TF32>, Cfg::SMEM, attr_done, p->ctx->device);
    if (rc) return rc;
    const int ld = p->Nv_pad;
    const int nbm = ld / TC_M, nbn = (B + 255) / 256, npp = (nbm + 1) / 2;
    long ntiles = 0;
    for (int P = 0; P < npp; ++P) {
        const int span = 2 * nbm - 4 * P;
        ntiles += (long)(kc > 0 ? (span + 2 * kc - 1) / (2 * kc) : 1) * nbn;
    }
    const int npairs = (int)std::min<long>(ntiles, max_pairs(p));
    const PairTile* work = nullptr;
    const int* starts = nullptr;
    const int* pslot = nullptr;
    rc = pair_schedule(p->sched, p->ctx->stream, nbm, nbn, 1, kc, TF32 ? 4 : 2, npairs, &work, &starts, &pslot);
    if (rc) return rc;
    goac::KTimer kt(p->ctx, goac::KID_SCORE_TC, p->ctx->stream);
    goac::launch_pdl(k_score_tc_pair<T, TF32>, 2 * npairs, 192, Cfg::SMEM, p->ctx->stream, mq, mj, work, starts, ld,
                     (const void*)p->qt.ptr, part, Bpad, p->ctx->d_err);
    GOAC_LAUNCH_CHECK("k_score_tc_pair");
    return GOAC_OK;
}

}  // namespace

namespace goac {

static goac_status prepare_split(goac_problem* p, int precision)
{
    const long n = (long)p->Nv_pad * p->Nv_pad;
    cudaStream_t st = p->ctx->stream;
    const int blocks = (int)std::min<long>((n + 255) / 256, 65535L * 4);
    if (precision == GOAC_PREC_BF16X2 || precision == GOAC_PREC_BF16X3) {
        if (!p->J_bf16) {
            GOAC_CUDA(cudaMalloc(&p->J_bf16, sizeof(__nv_bfloat16) * 3 * (size_t)n));
            goac::launch(k_split_bf16, blocks, 256, 0, st, p->J_vv, n, p->Nv_pad, p->J_bf16);
            GOAC_LAUNCH_CHECK("k_split_bf16");
        }
    } else {
        if (!p->J_tf32) {
            GOAC_CUDA(cudaMalloc(&p->J_tf32, sizeof(float) * 2 * (size_t)n));
            goac::launch(k_split_tf32, blocks, 256, 0, st, p->J_vv, n, p->Nv_pad, p->J_tf32);
            GOAC_LAUNCH_CHECK("k_split_tf32");
        }
    }
    return GOAC_OK;
}

goac_status prepare_f32(goac_problem* p)
{
    if (p->J_f32) return GOAC_OK;
    const long n = (long)p->Nv_pad * p->Nv_pad;
    GOAC_CUDA(cudaMalloc(&p->J_f32, sizeof(float) * (size_t)n));
    GOAC_CUDA(cudaMalloc(&p->diag_f32, sizeof(float) * (size_t)p->Nv));
    const int blocks = (int)std::min<long>((n + 255) / 256, 65535L * 4);
    goac::launch(k_copy_f32, blocks, 256, 0, p->ctx->stream, p->J_vv, n, p->J_f32, p->diag, p->Nv, p->diag_f32);
    GOAC_LAUNCH_CHECK("k_copy_f32");
    return GOAC_OK;
}

// Phi[b][v] (FP32, Bpad x Nv_pad) = sum_w J_vv[v][w] q[b][w] for real q given as
// hi / lo planes qt2 = [2][Bpad][Nv_pad], TF32 in FP32 storage (f16: FP16), on tcgen05.
goac_status phi_tc(goac_problem* p, const void* qt2, int Bpad, float* Phi, bool f16, int qshift)
{
    const int ld = p->Nv_pad;
    const long n = (long)ld * ld;
    cudaStream_t st = p->ctx->stream;
    const int blocks = (int)std::min<long>((n + 255) / 256, 65535L * 4);
    CUtensorMap ma, mb;
    goac_status rc = GOAC_OK;
    if (f16) {
        if (!p->J_f16_full) {
            GOAC_CUDA(cudaMalloc(&p->f16_exp, sizeof(int) * (ld / TC_M)));
            GOAC_CUDA(cudaMalloc(&p->J_f16_full, sizeof(__half) * 2 * (size_t)n));
            goac::launch(k_panel_exp, ld / TC_M, 256, 0, st, (const double*)p->J_vv, ld, 0, p->f16_exp);
            goac::launch(k_split_f16_full, blocks, 256, 0, st, (const double*)p->J_vv, ld, (const int*)p->f16_exp,
                         p->J_f16_full);
            GOAC_LAUNCH_CHECK("k_split_f16_full");
        }
        rc = make_map(&ma, p->J_f16_full, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, 2L * ld, ld, TC_M, PT_ROW);
        if (!rc) rc = make_map(&mb, (void*)qt2, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, 2L * Bpad, ld, PT_N, PT_ROW);
    } else {
        if (!p->J_tf32_full) {
            GOAC_CUDA(cudaMalloc(&p->J_tf32_full, sizeof(float) * 2 * (size_t)n));
            goac::launch(k_split_tf32_full, blocks, 256, 0, st, (const double*)p->J_vv, n, p->J_tf32_full);
            GOAC_LAUNCH_CHECK("k_split_tf32_full");
        }
        rc = make_map(&ma, p->J_tf32_full, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ld, 2L * ld, ld, TC_M, PT_ROW);
        if (!rc) rc = make_map(&mb, (void*)qt2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ld, 2L * Bpad, ld, PT_N, PT_ROW);
    }
    if (rc) return rc;
    static std::atomic<uint64_t> attr_tf32{0}, attr_f16{0};
    rc = f16 ? smem_attr_once((const void*)k_phi_tc<true>, PT_SMEM, attr_f16, p->ctx->device)
             : smem_attr_once((const void*)k_phi_tc<false>, PT_SMEM, attr_tf32, p->ctx->device);
    if (rc) return rc;
    if (Bpad % PT_N != 0) return fail(GOAC_ERR_INTERNAL, "phi_tc: padded batch must be a multiple of 256");
    const int nbn = Bpad / PT_N;
    const int ntiles = (ld / TC_M) * nbn;
    const int grid = std::min(ntiles, p->ctx->num_sms);
    // whole waves of whole tiles; the rest split in k-halves when that keeps them within one wave
    const int rest = ntiles % grid;
    const int nkb = ld / (f16 ? 32 : PT_KB);
    const int nfull = (rest > 0 && 2 * rest <= grid && nkb >= 2) ? ntiles - rest : ntiles;
    const int nitems = nfull + 2 * (ntiles - nfull);
    if (nitems > nfull) GOAC_CUDA(cudaMemsetAsync(Phi, 0, sizeof(float) * (size_t)Bpad * ld, st));
    KTimer kt(p->ctx, KID_SCORE_TC, st);
    if (f16)
        goac::launch(k_phi_tc<true>, grid, 192, PT_SMEM, st, ma, mb, nitems, nfull, nbn, nkb, ld, Bpad,
                     (const int*)p->f16_exp, qshift, Phi, p->ctx->d_err);
    else
        goac::launch(k_phi_tc<false>, grid, 192, PT_SMEM, st, ma, mb, nitems, nfull, nbn, nkb, ld, Bpad,
                     (const int*)nullptr, 0, Phi, p->ctx->d_err);
    GOAC_LAUNCH_CHECK("k_phi_tc");
    return GOAC_OK;
}

// Charge scaling of the exact form: the smallest kq <= 4 with every species
// charge times 2^kq an integer (-1: none), and the digit layout: r = 10 bits,
// T = 5 digits when 2^9 max|q 2^kq| Nv_pad < 2^24, else r = 8, T = 6 when
// 2^7 max|q 2^kq| Nv_pad < 2^24 (-2: neither), so that every digit sum of the
// tensor-core contraction is an integer below 2^24.
static int exact_layout(const goac_problem* p, int* r_out, int* T_out)
{
    for (int k = 0; k <= 4; ++k) {
        bool ok = true;
        double qmax = 0.0;
        for (double zz : p->z) {
            const double v = ldexp(zz, k);
            if (v != rint(v)) ok = false;
            qmax = std::max(qmax, fabs(v));
        }
        if (!ok) continue;
        const double bound = qmax * (double)p->Nv_pad;
        if (512.0 * bound < 16777216.0) {
            if (r_out) *r_out = 10;
            if (T_out) *T_out = 5;
        } else if (128.0 * bound < 16777216.0) {
            if (r_out) *r_out = 8;
            if (T_out) *T_out = 6;
        } else {
            return -2;
        }
        return k;
    }
    return -1;
}

bool exact_supported(goac_problem* p) { return exact_layout(p, nullptr, nullptr) >= 0; }

goac_status exact_info(const goac_problem* p, int32_t* digit_bits, int32_t* digits, int32_t* charge_shift)
{
    int r = 0, T = 0;
    const int kq = exact_layout(p, &r, &T);
    if (kq == -1) return fail(GOAC_ERR_UNSUPPORTED, "exact form: species charges are not multiples of 1/16");
    if (kq == -2) return fail(GOAC_ERR_UNSUPPORTED, "exact form: 128 max|q| Nv exceeds 2^24");
    if (digit_bits) *digit_bits = r;
    if (digits) *digits = T;
    if (charge_shift) *charge_shift = kq;
    return GOAC_OK;
}

static goac_status exact_charges(goac_problem* p)
{
    if (p->zq_dev) return GOAC_OK;
    int r = 0, T = 0;
    const int kq = exact_layout(p, &r, &T);
    if (kq == -1) return fail(GOAC_ERR_UNSUPPORTED, "exact form: species charges are not multiples of 1/16");
    if (kq == -2)
        return fail(GOAC_ERR_UNSUPPORTED, "exact form: 128 max|q| Nv exceeds 2^24 (digit sums would not be exact in FP32)");
    std::vector<double> zq(64, 0.0);
    for (int s2 = 0; s2 < p->S; ++s2) zq[s2] = ldexp(p->z[s2], kq);
    GOAC_CUDA(cudaMalloc(&p->zq_dev, sizeof(double) * 64));
    GOAC_CUDA(cudaMemcpy(p->zq_dev, zq.data(), sizeof(double) * 64, cudaMemcpyHostToDevice));
    p->dig_kq = kq;
    p->dig_r = r;
    p->dig_T = T;
    // |Phi| <= 2^(r-1) max|q| Nv_pad (a digit times at most Nv_pad charges), so a warp's sum of
    // 32 products q Phi stays inside int32 when 32 max|q|^2 2^(r-1) Nv_pad < 2^31
    double qmax = 0.0;
    for (int s2 = 0; s2 < p->S; ++s2) qmax = std::max(qmax, fabs(zq[s2]));
    p->dig_split = !(32.0 * qmax * qmax * ldexp(1.0, r - 1) * (double)p->Nv_pad < 2147483648.0);
    return GOAC_OK;
}

// Digits and panel exponents of the symmetric operand (sym) or of J_vv itself.
static goac_status build_digits(goac_problem* p, bool sym, __half** dig, int** pexp)
{
    goac_status rc = exact_charges(p);
    if (rc) return rc;
    const int ld = p->Nv_pad;
    const long n = (long)ld * ld;
    GOAC_CUDA(cudaMalloc(pexp, sizeof(int) * (ld / TC_M)));
    GOAC_CUDA(cudaMalloc(dig, sizeof(__half) * p->dig_T * (size_t)n));
    cudaStream_t st = p->ctx->stream;
    goac::launch(k_panel_exp, ld / TC_M, 256, 0, st, (const double*)p->J_vv, ld, sym ? 1 : 0, *pexp);
    const int blocks = (int)std::min<long>((n + 255) / 256, 65535L * 4);
    goac::launch(k_split_digits, blocks, 256, 0, st, (const double*)p->J_vv, ld, sym ? 1 : 0, (const int*)*pexp,
                 p->dig_r, p->dig_T, *dig);
    GOAC_LAUNCH_CHECK("exact digits");
    return GOAC_OK;
}

static goac_status prepare_exact(goac_problem* p)
{
    if (p->J_dig) return GOAC_OK;
    return build_digits(p, true, &p->J_dig, &p->dig_exp);
}

goac_status phi_exact(goac_problem* p, const int8_t* species, int B, double* E_out, void* phi_out, bool phi_f32)
{
    if (!p->J_dig_full) {
        goac_status rc = build_digits(p, false, &p->J_dig_full, &p->dig_exp_full);
        if (rc) return rc;
    }
    const int ld = p->Nv_pad;
    const int T = p->dig_T;
    const int Bpad = ((B + TC_N - 1) / TC_N) * TC_N;
    const int nbm = ld / TC_M, nbn = Bpad / TC_N;
    goac_status rc = ensure(p->qt, (size_t)Bpad * ld * 2);
    if (!rc) rc = ensure(p->phi_dig, sizeof(int) * (size_t)T * Bpad * ld);
    if (rc) return rc;
    cudaStream_t st = p->ctx->stream;
    goac::launch(k_make_qt<__half>, Bpad, MQ_T, 0, st, species, B, p->Nv, (const double*)p->zq_dev,
                 (const double*)p->z_dev, ld, (__half*)p->qt.ptr, (const double*)nullptr, (double*)nullptr, (void*)nullptr, 0);
    GOAC_LAUNCH_CHECK("k_make_qt (exact potentials)");
    CUtensorMap ma, mb;
    rc = make_map(&ma, p->J_dig_full, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, (long)T * ld, ld, TC_M);
    if (!rc) rc = make_map(&mb, p->qt.ptr, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, Bpad, ld, TC_N);
    if (rc) return rc;
    static std::atomic<uint64_t> attr_done{0};
    rc = smem_attr_once((const void*)k_phi_exact, EX_SMEM, attr_done, p->ctx->device);
    if (rc) return rc;
    const int ntiles = nbm * nbn * T;
    const int grid = std::min(ntiles, p->ctx->num_sms);
    {
        KTimer kt(p->ctx, KID_SCORE_TC, st);
        goac::launch(k_phi_exact, grid, 192, EX_SMEM, st, ma, mb, ntiles, nbm, ld / 64, ld, Bpad, T,
                     (int*)p->phi_dig.ptr, p->ctx->d_err);
        GOAC_LAUNCH_CHECK("k_phi_exact");
    }
    if (phi_f32)
        goac::launch(k_phi_exact_finish<float>, B, 256, 0, st, (const int*)p->phi_dig.ptr, Bpad, ld, p->Nv,
                     (const int*)p->dig_exp_full, p->dig_kq, p->dig_r, T, (const double*)p->phifix, species,
                     (const double*)p->z_dev, p->E_const, (float*)phi_out, E_out);
    else
        goac::launch(k_phi_exact_finish<double>, B, 256, 0, st, (const int*)p->phi_dig.ptr, Bpad, ld, p->Nv,
                     (const int*)p->dig_exp_full, p->dig_kq, p->dig_r, T, (const double*)p->phifix, species,
                     (const double*)p->z_dev, p->E_const, (double*)phi_out, E_out);
    GOAC_LAUNCH_CHECK("k_phi_exact_finish");
    return GOAC_OK;
}

// Tile shape of the scoring kernels for (precision, padded batch): the one
// goac_score_autotune or goac_score_set_shape stored, else whole panel ranges
// in tiles of 256 sites x 256 configurations on CTA pairs for the exact and
// BF16 forms and of 128 sites x 256 configurations for the TF32 forms.
static void pick_shape(const goac_problem* p, int precision, int Bpad, int* TM, int* TN, int* kc)
{
    const auto it = p->tile_shape.find(std::make_pair(precision, Bpad));
    const bool has = it != p->tile_shape.end();
    const bool pairs = precision == GOAC_PREC_EXACT || precision == GOAC_PREC_BF16X2 || precision == GOAC_PREC_BF16X3;
    *TM = has ? std::get<0>(it->second) : (pairs ? 2 * TC_M : TC_M);
    *TN = has ? std::get<1>(it->second) : TC_N;
    *kc = has ? std::get<2>(it->second) : 0;
}

static goac_status score_exact(goac_problem* p, const int8_t* species, int B, double* E_out)
{
    goac_status rc = prepare_exact(p);
    if (rc) return rc;
    const int ld = p->Nv_pad;
    const int T = p->dig_T;
    const int Bpad = ((B + TC_N - 1) / TC_N) * TC_N;
    const int nbm = ld / TC_M;
    int TM = 0, TN = 0, kc = 0;
    pick_shape(p, GOAC_PREC_EXACT, Bpad, &TM, &TN, &kc);
    const bool pair = TM == 2 * TC_M && TN == TC_N;
    const bool ct = TM == 2 * TC_M && TN == TC_NS;      // configurations on the TMEM lanes
    const bool split = p->dig_split;
    const int qbytes = ct || pair ? (split ? 2 : 1) : 0;    // the configuration-lane epilogues' charges
    const int nslots = pair || ct ? pair_slot_count(nbm, kc) : tc_tile_count(nbm, (B + TN - 1) / TN, T, kc).y;
    rc = ensure(p->qt, (size_t)Bpad * ld * 2);
    if (!rc && qbytes) rc = ensure(p->qi, (size_t)Bpad * ld * qbytes);
    if (!rc) rc = ensure(p->partial, sizeof(double) * ((size_t)nslots * T * Bpad + Bpad));
    if (rc) return rc;
    cudaStream_t st = p->ctx->stream;
    double* part = (double*)p->partial.ptr;
    double* lin = p->has_fixed ? part + (size_t)nslots * T * Bpad : nullptr;
    goac::launch(k_make_qt<__half>, Bpad, MQ_T, 0, st, species, B, p->Nv, (const double*)p->zq_dev,
                 (const double*)p->z_dev, ld, (__half*)p->qt.ptr,
                 (const double*)(p->has_fixed ? p->phifix : nullptr), lin, qbytes ? p->qi.ptr : nullptr, qbytes);
    GOAC_LAUNCH_CHECK("k_make_qt (exact)");
    CUtensorMap ma, mb;
    if (ct) {
        CUtensorMap mj, mjn;
        rc = make_map(&ma, p->qt.ptr, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, Bpad, ld, CT_M);
        if (!rc) rc = make_map(&mj, p->J_dig, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, (long)T * ld, ld, CT_N);
        if (!rc) rc = make_map(&mjn, p->J_dig, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, (long)T * ld, ld, CT_N / 2);
        if (rc) return rc;
        return split ? launch_exact_ct<true>(p, ma, mj, mjn, Bpad, B, kc, part, lin, E_out)
                     : launch_exact_ct<false>(p, ma, mj, mjn, Bpad, B, kc, part, lin, E_out);
    }
    if (pair) {
        // M: each CTA's 128 configurations of Q^T; N: each CTA's 128 digit rows of J'
        rc = make_map(&ma, p->qt.ptr, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, Bpad, ld, PX_HN);
        if (!rc) rc = make_map(&mb, p->J_dig, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, (long)T * ld, ld, TC_M);
    } else {
        rc = make_map(&ma, p->J_dig, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, (long)T * ld, ld, TC_M);
        if (!rc) rc = make_map(&mb, p->qt.ptr, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ld, Bpad, ld, TN);
    }
    if (rc) return rc;
    if (pair)
        return split ? launch_exact_pair<true>(p, ma, mb, Bpad, B, kc, part, lin, E_out)
                     : launch_exact_pair<false>(p, ma, mb, Bpad, B, kc, part, lin, E_out);
    if (TN == TC_NS)
        return split ? launch_exact<TC_NS, true>(p, ma, mb, Bpad, B, kc, part, lin, E_out)
                     : launch_exact<TC_NS, false>(p, ma, mb, Bpad, B, kc, part, lin, E_out);
    return split ? launch_exact<TC_N, true>(p, ma, mb, Bpad, B, kc, part, lin, E_out)
                 : launch_exact<TC_N, false>(p, ma, mb, Bpad, B, kc, part, lin, E_out);
}

template <int TN>
static goac_status launch_split(goac_problem* p, int precision, const CUtensorMap& ma, const CUtensorMap& mb,
                                int Bpad, int B, int kc, double* part)
{
    switch (precision) {
        case GOAC_PREC_TF32: return launch_tc<1, true, TN>(p, ma, mb, Bpad, B, kc, p->qt.ptr, part);
        case GOAC_PREC_TF32X2: return launch_tc<2, true, TN>(p, ma, mb, Bpad, B, kc, p->qt.ptr, part);
        case GOAC_PREC_BF16X2: return launch_tc<2, false, TN>(p, ma, mb, Bpad, B, kc, p->qt.ptr, part);
        case GOAC_PREC_BF16X3: return launch_tc<3, false, TN>(p, ma, mb, Bpad, B, kc, p->qt.ptr, part);
        default: return fail(GOAC_ERR_INVALID_ARG, "score_tc: bad precision");
    }
}

goac_status score_tc(goac_problem* p, const int8_t* species, int B, int precision, double* E_out)
{
    if (precision == GOAC_PREC_EXACT) return score_exact(p, species, B, E_out);
    goac_status rc = prepare_split(p, precision);
    if (rc) return rc;
    const bool tf32 = precision == GOAC_PREC_TF32 || precision == GOAC_PREC_TF32X2;
    const int ld = p->Nv_pad;
    const int Bpad = ((B + TC_N - 1) / TC_N) * TC_N;
    const int eb = tf32 ? 4 : 2;
    int TM = 0, TN = 0, kc = 0;
    pick_shape(p, precision, Bpad, &TM, &TN, &kc);
    const bool pair = TM == 2 * TC_M;       // on CTA pairs
    const int nslots = pair ? pair_slot_count(ld / TC_M, kc) : tc_tile_count(ld / TC_M, (B + TN - 1) / TN, 1, kc).y;
    rc = ensure(p->qt, (size_t)Bpad * ld * eb);
    if (!rc) rc = ensure(p->partial, sizeof(double) * ((size_t)nslots * Bpad + Bpad));
    if (rc) return rc;
    cudaStream_t st = p->ctx->stream;
    double* lin = p->has_fixed ? (double*)p->partial.ptr + (size_t)nslots * Bpad : nullptr;
    {
        const double* pf = p->has_fixed ? p->phifix : nullptr;
        if (tf32)
            goac::launch(k_make_qt<float>, Bpad, MQ_T, 0, st, species, B, p->Nv, (const double*)p->z_dev,
                         (const double*)p->z_dev, ld, (float*)p->qt.ptr, pf, lin, (void*)nullptr, 0);
        else
            goac::launch(k_make_qt<__nv_bfloat16>, Bpad, MQ_T, 0, st, species, B, p->Nv, (const double*)p->z_dev,
                         (const double*)p->z_dev, ld, (__nv_bfloat16*)p->qt.ptr, pf, lin, (void*)nullptr, 0);
        GOAC_LAUNCH_CHECK("k_make_qt");
    }
    CUtensorMap ma, mb;
    const int terms_alloc = tf32 ? 2 : 3;
    void* abase = tf32 ? (void*)p->J_tf32 : (void*)p->J_bf16;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    rc = make_map(&ma, abase, dt, eb, ld, (long)terms_alloc * ld, ld, TC_M);
    if (!rc) rc = make_map(&mb, p->qt.ptr, dt, eb, ld, Bpad, ld, pair ? PX_HN : TN);
    if (rc) return rc;
    double* part = (double*)p->partial.ptr;
    if (pair) {  // M: each CTA's 128 configurations of Q^T; N: each CTA's 128 rows of every term of J'
        switch (precision) {
            case GOAC_PREC_TF32: rc = launch_tc_pair<1, true>(p, mb, ma, Bpad, B, kc, part); break;
            case GOAC_PREC_TF32X2: rc = launch_tc_pair<2, true>(p, mb, ma, Bpad, B, kc, part); break;
            case GOAC_PREC_BF16X3: rc = launch_tc_pair<3, false>(p, mb, ma, Bpad, B, kc, part); break;
            default: rc = launch_tc_pair<2, false>(p, mb, ma, Bpad, B, kc, part); break;
        }
    } else
        rc = TN == TC_NS ? launch_split<TC_NS>(p, precision, ma, mb, Bpad, B, kc, part)
                         : launch_split<TC_N>(p, precision, ma, mb, Bpad, B, kc, part);
    if (rc) return rc;
    goac::launch_pdl(k_finish_tc, (B + 255) / 256, 256, 0, st, part, nslots, Bpad, B, p->E_const, lin, E_out);
    GOAC_LAUNCH_CHECK("k_finish_tc");
    return GOAC_OK;
}

// Tensor-core forms whose tile shape can be chosen.
static bool shaped_form(int precision)
{
    return precision == GOAC_PREC_TF32 || precision == GOAC_PREC_TF32X2 || precision == GOAC_PREC_BF16X2 ||
           precision == GOAC_PREC_BF16X3 || precision == GOAC_PREC_EXACT;
}

}  // namespace goac

extern "C" goac_status goac_score_set_shape(goac_problem* p, int32_t precision, int32_t B, int32_t tile_m,
                                            int32_t tile_n, int32_t ksplit)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_set_shape: NULL problem");
    if (!goac::shaped_form(precision))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_set_shape: not a tensor-core form");
    if (B < 1 || B > GOAC_MAX_BATCH || !(tile_m == 0 || tile_m == 128 || tile_m == 256) ||
        !(tile_n == 0 || tile_n == 128 || tile_n == 256) || ksplit < 0 || ksplit > 65535)
        return goac::fail(GOAC_ERR_INVALID_ARG,
                          "goac_score_set_shape: B >= 1, tile_m 0, 128 or 256, tile_n 0, 128 or 256, ksplit 0..65535");
    if (tile_m == 256 && precision != GOAC_PREC_EXACT && tile_n == 128)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_set_shape: 256 x 128 tiles need EXACT");
    const int Bpad = ((B + 255) / 256) * 256;
    const auto key = std::make_pair((int)precision, Bpad);
    if (tile_m == 0 && tile_n == 0 && ksplit == 0) p->tile_shape.erase(key);
    else p->tile_shape[key] = std::make_tuple(tile_m == 0 ? 128 : (int)tile_m, tile_n == 0 ? 256 : (int)tile_n, (int)ksplit);
    return GOAC_OK;
}

extern "C" goac_status goac_score_autotune(goac_problem* p, const int8_t* species_dev, int32_t B, int32_t precision,
                                           int32_t* tile_m_out, int32_t* tile_n_out, int32_t* ksplit_out,
                                           double* ms_out)
{
    if (!p || !species_dev || B < 1 || B > GOAC_MAX_BATCH)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_autotune: bad argument");
    if (!goac::shaped_form(precision))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_autotune: not a tensor-core form");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    cudaStream_t st = p->ctx->stream;
    double* E = nullptr;
    GOAC_CUDA(cudaMalloc(&E, sizeof(double) * (size_t)B));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int nbm = p->Nv_pad / 128;
    const int Bpad = ((B + 255) / 256) * 256;
    const auto key = std::make_pair((int)precision, Bpad);
    // candidates: {tile_m, tile_n} x k-chunks; 256-site tiles on CTA pairs for every form, and the one-CTA
    // configuration-lane tiles for the exact form
    const int shapes[4][2] = {{128, 256}, {128, 128}, {256, 256}, {256, 128}};
    const int nshapes = precision == GOAC_PREC_EXACT ? 4 : 3;
    const int kcs[5] = {0, 16, 8, 4, 2};
    int best_tm = 0, best_tn = 0, best_kc = 0;
    float best = 0.0f;
    goac_status rc = GOAC_OK;
    for (int i = 0; i < nshapes && !rc; ++i)
        for (int j = 0; j < 5 && !rc; ++j) {
            if (kcs[j] >= nbm) continue;                 // the same as whole panel ranges
            p->tile_shape[key] = std::make_tuple(shapes[i][0], shapes[i][1], kcs[j]);
            rc = goac_score(p, species_dev, B, precision, E);     // schedule, operands, warm-up
            if (rc) break;
            cudaEventRecord(a, st);
            for (int r = 0; r < 3 && !rc; ++r) rc = goac_score(p, species_dev, B, precision, E);
            cudaEventRecord(b, st);
            if (rc) break;
            cudaEventSynchronize(b);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (best_tn == 0 || ms < best) {
                best_tm = shapes[i][0];
                best_tn = shapes[i][1];
                best_kc = kcs[j];
                best = ms;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(st);
    cudaFree(E);
    if (rc) {
        p->tile_shape.erase(key);
        return rc;
    }
    p->tile_shape[key] = std::make_tuple(best_tm, best_tn, best_kc);
    if (tile_m_out) *tile_m_out = best_tm;
    if (tile_n_out) *tile_n_out = best_tn;
    if (ksplit_out) *ksplit_out = best_kc;
    if (ms_out) *ms_out = best / 3.0;
    rc = goac::check_device_error(p->ctx);
    return rc;
}
