// Batched scoring E_b = q_b^T J_vv q_b + 2 q_b . phi_fix + E_const on the
// tcgen05 tensor cores (sm_103a): the objective of Eq. 2 evaluated for a whole
// population as one dense contraction Phi = J_vv Q followed by a row-dot.
//
// J_vv is split into T low-precision terms (BF16: J = J1 + J2 [+ J3], each the
// BF16 rounding of the remainder; TF32: hi + lo).  Charges are small integers
// and exact in BF16 / TF32, so Q needs no split.  Per CTA one 128 (sites) x
// 256 (configs) FP32 accumulator lives in TMEM (256 columns); every k-block
// stage holds the T J-tiles (128 x 128 B each) and one Q-tile (256 x 128 B),
// loaded by TMA with the 128-byte swizzle, and the single MMA thread issues
// T x 4 tcgen05.mma (K = 16 BF16 / 8 TF32 each) into the same accumulator.
// Warp roles: warp 0 lane 0 = TMA producer, warp 1 lane 0 = MMA issuer,
// warp 2 = TMEM allocator; then all 4 warps run the epilogue: tcgen05.ld of
// their 32 TMEM lanes (= 32 sites), q (Phi + 2 phi_fix) in FP32, a butterfly
// transpose-reduce across the warp so lane l owns config column l, and the
// 4 warp sums are added in FP64 into partial[m-tile][config].  A second tiny
// kernel adds the m-tiles in a fixed order plus E_const (deterministic).
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int TC_M = 128;              // sites per tile (TMEM lanes)
constexpr int TC_N = 256;              // configurations per tile (TMEM columns)
constexpr int ROW_BYTES = 128;         // one k-block row: 64 BF16 or 32 FP32
constexpr int A_TILE = TC_M * ROW_BYTES;
constexpr int B_TILE = TC_N * ROW_BYTES;
constexpr long long WAIT_LIMIT = 4000000000LL;   // ~2 s of SM clock

template <int T>
struct TcCfg {
    static constexpr int STAGE = T * A_TILE + B_TILE;
    static constexpr int STAGES_RAW = (196 * 1024) / STAGE;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM = STAGES * STAGE + 1024 + BAR_BYTES;
};

template <int T, bool TF32>
__global__ void __launch_bounds__(128, 1)
    k_score_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int nkb,
               int Nv_pad, int Nv, const void* __restrict__ qt, int ldq, const double* __restrict__ phifix,
               double* __restrict__ partial, int Bpad, int* __restrict__ err)
{
    using Cfg = TcCfg<T>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr int STAGE = Cfg::STAGE;
    constexpr int KE = TF32 ? 32 : 64;          // elements per 128-byte row
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    __shared__ float red[4][TC_N];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TC_M;
    const int n0 = blockIdx.x * TC_N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            goacd::mbar_init(&full[s], 1);
            goacd::mbar_init(&empty[s], 1);
        }
        goacd::mbar_init(done, 1);
        *abort_flag = 0;
        goacd::fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        goacd::prefetch_tmap(&tmA);
        goacd::prefetch_tmap(&tmB);
    }
    if (warp == 2) {
        goacd::tmem_alloc(tmem_slot, TC_N);
        goacd::tmem_relinquish();
    }
    goacd::tc_fence_before();
    __syncthreads();
    goacd::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                const uint32_t use = (uint32_t)(kb / STAGES);
                if (kb >= STAGES && !goacd::mbar_wait_bounded(&empty[s], (use - 1) & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_PRODUCER, kb);
                    break;
                }
                if (*abort_flag) break;
                uint8_t* st = smem + s * STAGE;
                goacd::mbar_arrive_expect_tx(&full[s], STAGE);
#pragma unroll
                for (int t = 0; t < T; ++t) goacd::tma_load_2d(st + t * A_TILE, &tmA, &full[s], kb * KE, t * Nv_pad + m0);
                goacd::tma_load_2d(st + T * A_TILE, &tmB, &full[s], kb * KE, n0);
                issued = kb + 1;
            }
            if (*abort_flag) {
                // drain: every copy this thread started must land before the CTA exits
                for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
                    if (!goacd::mbar_wait_bounded(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1, WAIT_LIMIT))
                        goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_DRAIN, kb);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = goacd::idesc_f32acc(TF32 ? 2u : 1u, TC_M, TC_N);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                const uint32_t use = (uint32_t)(kb / STAGES);
                if (!goacd::mbar_wait_bounded(&full[s], use & 1, WAIT_LIMIT)) {
                    *abort_flag = 1;
                    goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_MMA, kb);
                    break;
                }
                if (*abort_flag) break;
                goacd::tc_fence_after();
                const uint32_t a0 = goacd::smem_u32(smem + s * STAGE);
                const uint32_t b0 = a0 + T * A_TILE;
#pragma unroll
                for (int t = 0; t < T; ++t)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = goacd::sdesc_k128(a0 + t * A_TILE + kk * 32);
                        const uint64_t bd = goacd::sdesc_k128(b0 + kk * 32);
                        const uint32_t acc = (kb | t | kk) != 0;
                        if (TF32) goacd::mma_tf32(tmem, ad, bd, idesc, acc);
                        else goacd::mma_bf16(tmem, ad, bd, idesc, acc);
                    }
                goacd::mma_commit(&empty[s]);
            }
            goacd::mma_commit(done);
        }
        __syncwarp();
    }

    // ---- epilogue: all four warps -------------------------------------------
    const bool ok = goacd::mbar_wait_bounded(done, 0, WAIT_LIMIT) && !*abort_flag;
    if (!ok && threadIdx.x == 0) goacd::report(err, GOAC_ERR_TIMEOUT, goac::SITE_TC_EPILOGUE, 0);
    goacd::tc_fence_after();
    if (ok) {
        const int row = warp * 32 + lane;
        const int v = m0 + row;
        const float pf2 = v < Nv ? (float)(2.0 * phifix[v]) : 0.0f;
#pragma unroll 1
        for (int c = 0; c < TC_N / 32; ++c) {
            uint32_t r[32];
            goacd::tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
            goacd::tmem_ld_wait();
            float val[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const long b = n0 + c * 32 + j;
                float q;
                if (TF32) q = ((const float*)qt)[b * ldq + v];
                else q = __bfloat162float(((const __nv_bfloat16*)qt)[b * ldq + v]);
                val[j] = q * (__uint_as_float(r[j]) + pf2);
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
            red[warp][c * 32 + lane] = val[0];
        }
    }
    goacd::tc_fence_before();
    __syncthreads();
    if (ok) {
        for (int col = threadIdx.x; col < TC_N; col += 128) {
            const double s = (double)red[0][col] + (double)red[1][col] + (double)red[2][col] + (double)red[3][col];
            partial[(long)blockIdx.y * Bpad + n0 + col] = s;
        }
    }
    if (warp == 2) {
        goacd::tc_fence_after();
        goacd::tmem_dealloc(tmem, TC_N);
    }
}

__global__ void k_split_bf16(const double* __restrict__ J, long n, __nv_bfloat16* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double x = J[e];
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

__global__ void k_split_tf32(const double* __restrict__ J, long n, float* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double x = J[e];
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

// Q^T[b][v] = z[species[b][v]] in BF16 or FP32, zero padded to Bpad x ld.
template <typename QT>
__global__ void k_make_qt(const int8_t* __restrict__ species, int B, int Nv, const double* __restrict__ z, int Bpad,
                          int ld, QT* __restrict__ qt)
{
    __shared__ float zs[64];
    if (threadIdx.x < 64) zs[threadIdx.x] = (float)z[threadIdx.x];
    __syncthreads();
    const long total = (long)Bpad * ld;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int b = (int)(e / ld), v = (int)(e % ld);
        float q = (b < B && v < Nv) ? zs[species[(long)b * Nv + v]] : 0.0f;
        if constexpr (sizeof(QT) == 2) qt[e] = __float2bfloat16(q);
        else qt[e] = q;
    }
}

__global__ void k_finish_tc(const double* __restrict__ partial, int mtiles, int Bpad, int B, double E_const,
                            double* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
    for (int m = 0; m < mtiles; ++m) s += partial[(long)m * Bpad + b];
    E[b] = s + E_const;
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

// 2D K-major tensor map: inner dim = `inner` elements (row pitch `pitch_elems`),
// outer dim = `rows`; box = 128 bytes x box_rows, 128-byte swizzle.
goac_status make_map(CUtensorMap* map, void* base, CUtensorMapDataType dt, int elem_bytes, long inner, long rows,
                     long pitch_elems, int box_rows)
{
    auto enc = get_encode();
    if (!enc) return goac::fail(GOAC_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    if (((uintptr_t)base & 15) != 0 || (pitch_elems * elem_bytes) % 16 != 0)
        return goac::fail(GOAC_ERR_INTERNAL, "tensor map base / pitch not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * elem_bytes)};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return goac::fail(GOAC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return GOAC_OK;
}

template <int T, bool TF32>
goac_status launch_tc(goac_problem* p, const CUtensorMap& ma, const CUtensorMap& mb, int Bpad, const void* qt,
                      double* part)
{
    using Cfg = TcCfg<T>;
    auto kern = k_score_tc<T, TF32>;
    static bool attr_set = false;
    if (!attr_set) {
        GOAC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        attr_set = true;
    }
    const int ld = p->Nv_pad;
    const int nkb = TF32 ? ld / 32 : ld / 64;
    dim3 grid(Bpad / TC_N, ld / TC_M);
    kern<<<grid, 128, Cfg::SMEM, p->ctx->stream>>>(ma, mb, nkb, ld, p->Nv, qt, ld, p->phifix, part, Bpad,
                                                   p->ctx->d_err);
    GOAC_LAUNCH_CHECK("k_score_tc");
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
            k_split_bf16<<<blocks, 256, 0, st>>>(p->J_vv, n, p->J_bf16);
            GOAC_LAUNCH_CHECK("k_split_bf16");
        }
    } else {
        if (!p->J_tf32) {
            GOAC_CUDA(cudaMalloc(&p->J_tf32, sizeof(float) * 2 * (size_t)n));
            k_split_tf32<<<blocks, 256, 0, st>>>(p->J_vv, n, p->J_tf32);
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
    k_copy_f32<<<blocks, 256, 0, p->ctx->stream>>>(p->J_vv, n, p->J_f32, p->diag, p->Nv, p->diag_f32);
    GOAC_LAUNCH_CHECK("k_copy_f32");
    return GOAC_OK;
}

goac_status score_tc(goac_problem* p, const int8_t* species, int B, int precision, double* E_out)
{
    goac_status rc = prepare_split(p, precision);
    if (rc) return rc;
    const bool tf32 = precision == GOAC_PREC_TF32 || precision == GOAC_PREC_TF32X2;
    const int ld = p->Nv_pad;
    const int Bpad = ((B + TC_N - 1) / TC_N) * TC_N;
    const int eb = tf32 ? 4 : 2;
    rc = ensure(p->qt, (size_t)Bpad * ld * eb);
    if (!rc) rc = ensure(p->partial, sizeof(double) * (size_t)(ld / TC_M) * Bpad);
    if (rc) return rc;
    cudaStream_t st = p->ctx->stream;
    {
        const long total = (long)Bpad * ld;
        const int blocks = (int)std::min<long>((total + 255) / 256, 65535L * 4);
        if (tf32) k_make_qt<float><<<blocks, 256, 0, st>>>(species, B, p->Nv, p->z_dev, Bpad, ld, (float*)p->qt.ptr);
        else k_make_qt<__nv_bfloat16><<<blocks, 256, 0, st>>>(species, B, p->Nv, p->z_dev, Bpad, ld,
                                                             (__nv_bfloat16*)p->qt.ptr);
        GOAC_LAUNCH_CHECK("k_make_qt");
    }
    CUtensorMap ma, mb;
    const int terms_alloc = tf32 ? 2 : 3;
    void* abase = tf32 ? (void*)p->J_tf32 : (void*)p->J_bf16;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    rc = make_map(&ma, abase, dt, eb, ld, (long)terms_alloc * ld, ld, TC_M);
    if (!rc) rc = make_map(&mb, p->qt.ptr, dt, eb, ld, Bpad, ld, TC_N);
    if (rc) return rc;
    double* part = (double*)p->partial.ptr;
    switch (precision) {
        case GOAC_PREC_TF32: rc = launch_tc<1, true>(p, ma, mb, Bpad, p->qt.ptr, part); break;
        case GOAC_PREC_TF32X2: rc = launch_tc<2, true>(p, ma, mb, Bpad, p->qt.ptr, part); break;
        case GOAC_PREC_BF16X2: rc = launch_tc<2, false>(p, ma, mb, Bpad, p->qt.ptr, part); break;
        case GOAC_PREC_BF16X3: rc = launch_tc<3, false>(p, ma, mb, Bpad, p->qt.ptr, part); break;
        default: return fail(GOAC_ERR_INVALID_ARG, "score_tc: bad precision");
    }
    if (rc) return rc;
    k_finish_tc<<<(B + 255) / 256, 256, 0, st>>>(part, ld / TC_M, Bpad, B, p->E_const, E_out);
    GOAC_LAUNCH_CHECK("k_finish_tc");
    return GOAC_OK;
}

}  // namespace goac
