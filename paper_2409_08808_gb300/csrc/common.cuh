// Internal definitions shared by the CUDA translation units of libgoac.
// Device-side helpers: Philox4x32-10 (SC'11), bounded mbarrier waits, and
// thin inline-PTX wrappers for TMA, mbarrier and tcgen05 (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/goac.h"

// ---------------------------------------------------------------------------
// Host-side error plumbing
// ---------------------------------------------------------------------------
namespace goac {

void set_error(const std::string& msg);
goac_status fail(goac_status code, const std::string& msg);
goac_status cuda_fail(cudaError_t e, const char* what);

#define GOAC_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e__ = (call);                                    \
        if (e__ != cudaSuccess) return goac::cuda_fail(e__, #call);  \
    } while (0)

#define GOAC_LAUNCH_CHECK(what)                                      \
    do {                                                             \
        cudaError_t e__ = cudaGetLastError();                        \
        if (e__ != cudaSuccess) return goac::cuda_fail(e__, what);   \
    } while (0)

// Device error word layout: [0] = first error code (goac_status), [1] = site id,
// [2] = extra info, [3] = count of errors.
enum DevErrSite : int {
    SITE_TC_PRODUCER = 1,
    SITE_TC_MMA = 2,
    SITE_TC_EPILOGUE = 3,
    SITE_TC_DRAIN = 4,
    SITE_MC = 10,
    SITE_GA = 20,
    SITE_ROUND = 30,
};

}  // namespace goac

// A device-resident growable buffer owned by a context or problem.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct goac_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int* d_err = nullptr;          // 4 ints, see DevErrSite
    DevBuf host_io_species;        // device staging for goac_score_host
    DevBuf host_io_E;
    void* pinned = nullptr;        // not used by the stream path; reserved
    // pipelined host-buffer scoring (goac_score_host_async): two staging slots
    cudaStream_t copy_stream = nullptr;
    DevBuf async_species[2];
    DevBuf async_E[2];
    cudaEvent_t async_h2d[2] = {nullptr, nullptr};    // slot's species copy landed
    cudaEvent_t async_done[2] = {nullptr, nullptr};   // slot's scoring and E copy finished
    bool async_used[2] = {false, false};
    int async_next = 0;
    // per-kernel event timing (goac_ctx_set_timing / goac_ctx_kernel_time)
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed[8];
    std::vector<cudaEvent_t> event_pool;
    // batched-MC graph cache
    cudaGraphExec_t batch_graph = nullptr;
    uint64_t batch_graph_key = 0;
    DevBuf batch_desc;
    DevBuf batch_items;
    DevBuf batch_counter;
    DevBuf ga_dev;                 // batched GA: device copy of the population entries
};

// A persistent scoring kernel's tile schedule on the device (tiles, per-CTA
// starts, per-panel partial-slot starts) and the shape it was built for.
struct TcSched {
    DevBuf buf;
    uint64_t key[2] = {0, 0};
    int ntiles = 0, nslots = 0, grid = 0;
};

// Per-problem data on the device.  Kernels receive the plain pointers.
struct goac_problem {
    goac_ctx* ctx = nullptr;
    int N = 0, Nv = 0, S = 0, ncls = 0;
    int Nv_pad = 0;            // multiple of 128 (tensor-core tiles)
    bool has_fixed = false;    // any fixed ion (phi_fix may be non-zero)
    double E_const = 0.0;
    // host copies
    std::vector<int32_t> vclass, cls_start, cls_pos, counts;
    std::vector<double> z;
    std::vector<uint32_t> wprefix;
    uint32_t wtotal = 0;
    int nmovable = 0, only_movable = -1;
    // device copies
    double* J_vv = nullptr;    // Nv_pad x Nv_pad FP64, zero padded
    double* diag = nullptr;    // Nv   (J_vv diagonal)
    double* phifix = nullptr;  // Nv_pad (zero padded)
    float* phifix_f32 = nullptr;  // Nv_pad, phifix rounded to FP32 (relaxed-gradient chain rule)
    double* z_dev = nullptr;   // S
    int32_t* vclass_dev = nullptr;
    int32_t* cls_start_dev = nullptr;
    int32_t* cls_pos_dev = nullptr;
    int32_t* cls_rank_dev = nullptr;   // Nv: index p of each variable site in cls_pos
    int32_t* counts_dev = nullptr;
    uint32_t* wprefix_dev = nullptr;
    // lazily built operand copies for the tensor-core and FP32 paths
    __nv_bfloat16* J_bf16 = nullptr;   // [3][Nv_pad][Nv_pad]
    float* J_tf32 = nullptr;           // [2][Nv_pad][Nv_pad] (hi, lo) of the symmetric operand
    float* J_tf32_full = nullptr;      // [2][Nv_pad][Nv_pad] (hi, lo) of J_vv itself
    __half* J_f16_full = nullptr;      // [2][Nv_pad][Nv_pad] (hi, lo) of J_vv 2^(15 - e_I), FP16
    int* f16_exp = nullptr;            // e_I per 128-row panel of J_vv (max |J| < 2^e_I)
    float* J_f32 = nullptr;            // Nv_pad x Nv_pad (MC / GA FP32 variant)
    float* diag_f32 = nullptr;
    // scoring scratch
    DevBuf qt, partial, phi, score_tmp, topk_tmp, grad_tmp;
    DevBuf qi;                 // exact form: integer charges beside Q^T (int8, or int16 when the digit sums split)
    DevBuf ga_incr;            // incremental GA rescoring: 2 x P x Nv potentials, P x 2 parents
    DevBuf ga_buf;             // GA: second population buffer, fitness sums, elite, stop states, parents
    DevBuf ga_dev;             // GA: device copy of the population entries
    int mc_tuned[2][2] = {{0, 0}, {0, 0}};   // [FP64, FP32]: autotuned {warps per chain, chains per CTA}, 0 = none
    // persistent tensor-core schedules (device copies) for the last shapes
    TcSched sched, sched_ex;
    // scoring tile shape per (precision, padded batch): {sites per tile (256: a CTA pair),
    // configurations per tile, k-chunk in 128-column blocks}
    std::map<std::pair<int, int>, std::tuple<int, int, int>> tile_shape;
    // exact form: FP16 digits of the symmetric operand, panel exponents, scaled charges
    __half* J_dig = nullptr;           // [dig_T][Nv_pad][Nv_pad]
    int* dig_exp = nullptr;            // Nv_pad / 128
    double* zq_dev = nullptr;          // 64, charges times 2^dig_kq
    int dig_kq = -1;
    int dig_r = 0, dig_T = 0;          // digit width (bits) and number of digits
    bool dig_split = true;             // epilogue splits each digit sum in 12-bit halves (else one int32 sum)
    // exact-form potentials: digits of J_vv itself, its panel exponents, digit sums
    __half* J_dig_full = nullptr;      // [dig_T][Nv_pad][Nv_pad]
    int* dig_exp_full = nullptr;       // Nv_pad / 128
    DevBuf phi_dig;                    // [dig_T][Bpad][Nv_pad] int32
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
namespace goacd {

// Philox4x32-10 counter-based generator (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_seed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    return philox(make_uint4(c0, c1, c2, c3), (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t draw_below(uint32_t x, uint32_t n)
{
    return __umulhi(x, n);
}

__device__ __forceinline__ void report(int* err, int code, int site, int info)
{
    if (err == nullptr) return;
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = site;
        err[2] = info;
    }
    atomicAdd(err + 3, 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, giving up after
// roughly `limit_cycles` SM clock cycles.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_cycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier among `count` threads (a multiple of 32) on hardware barrier `id` (1..15).
__device__ __forceinline__ void named_bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---- programmatic dependent launch -----------------------------------------------
// Wait until the preceding kernel in the stream has completed and its memory
// is visible (returns at once when the kernel was not launched as a dependent).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Allow the next kernel in the stream (if launched as a dependent) to start.
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- TMA ---------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- tcgen05 -----------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 or FP16 inputs, as the
// instruction descriptor says; FP32 accumulate).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Same for kind::tf32 (FP32 storage, TF32 inputs, FP32 accumulate).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread l of the warp receives its
// lane's 32 columns.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- CTA pairs (clusters of two, tcgen05 cta_group::2) ----------------------------
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// All threads of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on an mbarrier given by its shared::cluster address (possibly in the peer CTA).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Tensor memory of a CTA pair: one warp of each CTA of the pair takes part.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* smem_slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (+)= A * B^T over the CTA pair, kind::f16: rows 0..M/2-1 of A and D in the
// issuing (even) CTA, the rest in its peer at the same shared / tensor-memory
// offsets; B's first N/2 rows in the even CTA, the rest in the peer.
__device__ __forceinline__ void mma_f16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier at this offset in every CTA of cta_mask once the pair
// MMAs issued so far by this thread complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t cta_mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(cta_mask)
        : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on an
// mbarrier of the CTA pair (shared::cluster address, the even CTA's).
__device__ __forceinline__ void tma_load_2d_pair(void* smem_dst, const CUtensorMap* map, uint32_t mbar_cluster, int x,
                                                 int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar_cluster)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile whose rows are 128
// bytes, stored with the 128-byte swizzle (8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format fmt (kind::f16: 0 = FP16,
// 1 = BF16; kind::tf32: 2 = TF32), both K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_f32acc(uint32_t fmt, uint32_t M, uint32_t N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

}  // namespace goacd

// Every kernel launch of the library goes through launch(): it counts the
// launch (goac_launch_count) and returns the launch error.
namespace goac {
void count_launch();

template <typename... KArgs, typename... Args>
inline cudaError_t launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args&&... args)
{
    count_launch();
    kern<<<grid, block, smem, st>>>(static_cast<KArgs>(args)...);
    return cudaGetLastError();
}

// Same, as a programmatic dependent launch: the kernel may become resident while
// its predecessor in the stream is still running, and must execute
// goacd::pdl_wait() before it reads anything the predecessor writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args)
{
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Kernel families timed with CUDA events when timing is enabled on a context.
enum KernelId : int {
    KID_SCORE_TC = 0,   // tensor-core scoring main kernel
    KID_SCORE_CC = 1,   // CUDA-core (FP64 / FP32) scoring GEMM
    KID_MC = 2,         // Monte Carlo chains (single or batched)
    KID_GA = 3,         // GA children
    KID_EWALD_REAL = 4, // Ewald real-space pair kernel
    KID_EWALD_SYRK = 5, // Ewald reciprocal SYRK
    KID_GA_INCR = 6,    // incremental GA rescoring
    KID_COUNT = 8
};

// Records a CUDA event pair around the launches in its scope (no-op unless
// timing is enabled on the context).
struct KTimer {
    goac_ctx* ctx;
    int id;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(goac_ctx* c, int kid, cudaStream_t s);
    ~KTimer();
};
goac_status ensure(DevBuf& b, size_t bytes);
goac_status check_device_error(goac_ctx* ctx);
int tc_supported(goac_ctx* ctx);
// FP64 J.Q for a population: optional phi_out (B x Nv, phi = J_vv q + phi_fix)
// and/or energies (E = q.(J q + 2 phi_fix) + E_const).
goac_status score_f64(goac_problem* p, const int8_t* species, int B, double* E_out, double* phi_out);
goac_status score_f32(goac_problem* p, const int8_t* species, int B, double* E_out, float* phi_out);
goac_status score_tc(goac_problem* p, const int8_t* species, int B, int precision, double* E_out);
goac_status prepare_f32(goac_problem* p);
goac_status phi_tc(goac_problem* p, const void* qt2, int Bpad, float* Phi, bool f16 = false, int qshift = 0);
// Exact-form potentials and energies (phi = J_vv q + phi_fix, B x Nv FP64, and
// E as score_f64) on the tensor cores; false from exact_supported() means the
// charges do not admit the exact form and score_f64 must be used.
bool exact_supported(goac_problem* p);
goac_status exact_info(const goac_problem* p, int32_t* digit_bits, int32_t* digits, int32_t* charge_shift);
// phi_out: B x Nv FP64, or FP32 (rounded once from the FP64-grade value) when phi_f32.
goac_status phi_exact(goac_problem* p, const int8_t* species, int B, double* E_out, void* phi_out,
                      bool phi_f32 = false);
}  // namespace goac
