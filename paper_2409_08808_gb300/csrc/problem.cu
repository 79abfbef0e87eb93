// Context, errors, problem set-up (Eq. 2 with its constraints), the plain
// FP64 batched scoring path, random structures and top-k FP64 rescoring.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "common.cuh"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
namespace goac {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

goac_status fail(goac_status code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

goac_status cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GOAC_ERR_OOM : GOAC_ERR_CUDA;
}

goac_status ensure(DevBuf& b, size_t bytes)
{
    if (b.bytes >= bytes && b.ptr) return GOAC_OK;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
    b.bytes = want;
    return GOAC_OK;
}

goac_status check_device_error(goac_ctx* ctx)
{
    int h[4] = {0, 0, 0, 0};
    GOAC_CUDA(cudaMemcpyAsync(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    GOAC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h[0] != 0) {
        char buf[160];
        snprintf(buf, sizeof(buf), "device error %d at site %d (info %d, %d errors)", h[0], h[1], h[2], h[3]);
        GOAC_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream));
        return fail(h[0], buf);
    }
    return GOAC_OK;
}

static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

KTimer::KTimer(goac_ctx* c, int kid, cudaStream_t s) : ctx(c), id(kid), st(s)
{
    if (!ctx || !ctx->timing) return;
    auto take = [&]() {
        cudaEvent_t e = nullptr;
        if (!ctx->event_pool.empty()) {
            e = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    };
    a = take();
    b = take();
    cudaEventRecord(a, st);
}

KTimer::~KTimer()
{
    if (!a) return;
    cudaEventRecord(b, st);
    ctx->timed[id].push_back({a, b});
}

int tc_supported(goac_ctx* ctx)
{
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
    return major == 10 && minor == 3;
}

}  // namespace goac

extern "C" const char* goac_last_error(void) { return goac::g_last_error.c_str(); }

extern "C" int32_t goac_version(void) { return 100; }

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
extern "C" goac_status goac_ctx_create(int32_t device, void* stream, goac_ctx** out)
{
    if (!out) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    GOAC_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_create: bad device");
    GOAC_CUDA(cudaSetDevice(device));
    goac_ctx* c = new goac_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (!goac::tc_supported(c)) {
        delete c;
        return goac::fail(GOAC_ERR_UNSUPPORTED, "goac_ctx_create: device is not compute capability 10.3 (GB300)");
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->d_err, 4 * sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return goac::cuda_fail(e, "cudaMalloc(error word)");
    }
    cudaMemset(c->d_err, 0, 4 * sizeof(int));
    cudaDeviceSynchronize();
    *out = c;
    return GOAC_OK;
}

static void free_buf(DevBuf& b)
{
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

extern "C" goac_status goac_ctx_destroy(goac_ctx* ctx)
{
    if (!ctx) return GOAC_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    for (auto& v : ctx->timed)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    free_buf(ctx->host_io_species);
    free_buf(ctx->host_io_E);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (int s = 0; s < 2; ++s) {
        if (ctx->async_h2d[s]) cudaEventDestroy(ctx->async_h2d[s]);
        if (ctx->async_done[s]) cudaEventDestroy(ctx->async_done[s]);
        free_buf(ctx->async_species[s]);
        free_buf(ctx->async_E[s]);
    }
    free_buf(ctx->batch_desc);
    free_buf(ctx->batch_items);
    free_buf(ctx->batch_counter);
    free_buf(ctx->ga_dev);
    cudaFree(ctx->d_err);
    delete ctx;
    return GOAC_OK;
}

extern "C" goac_status goac_ctx_set_timing(goac_ctx* ctx, int32_t enable)
{
    if (!ctx) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_set_timing: ctx is NULL");
    ctx->timing = enable != 0;
    return GOAC_OK;
}

extern "C" goac_status goac_ctx_kernel_time(goac_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches)
{
    if (!ctx || kernel < 0 || kernel >= goac::KID_COUNT)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_kernel_time: bad argument");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    double tot = 0.0;
    int64_t n = 0;
    for (auto& pr : ctx->timed[kernel]) {
        GOAC_CUDA(cudaEventSynchronize(pr.second));
        float ms = 0.0f;
        GOAC_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
        ++n;
        ctx->event_pool.push_back(pr.first);
        ctx->event_pool.push_back(pr.second);
    }
    ctx->timed[kernel].clear();
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return GOAC_OK;
}

extern "C" int64_t goac_launch_count(void) { return (int64_t)goac::g_launches.load(); }

extern "C" goac_status goac_ctx_set_stream(goac_ctx* ctx, void* stream)
{
    if (!ctx) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_set_stream: ctx is NULL");
    ctx->stream = (cudaStream_t)stream;
    return GOAC_OK;
}

extern "C" goac_status goac_ctx_synchronize(goac_ctx* ctx)
{
    if (!ctx) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ctx_synchronize: ctx is NULL");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    if (ctx->copy_stream) GOAC_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    return goac::check_device_error(ctx);
}

// ---------------------------------------------------------------------------
// Problem set-up kernels
// ---------------------------------------------------------------------------
namespace {

__global__ void k_gather_jvv(const double* __restrict__ J, int N, const int32_t* __restrict__ vsite, int Nv,
                             int ld, double* __restrict__ Jvv, double* __restrict__ diag)
{
    long total = (long)ld * ld;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int a = (int)(e / ld), b = (int)(e % ld);
        double v = 0.0;
        if (a < Nv && b < Nv) v = J[(long)vsite[a] * N + vsite[b]];
        Jvv[e] = v;
        if (a == b && a < Nv) diag[a] = v;
    }
}

// s_i = sum_f J[i][f] q_f over fixed sites f; one warp per row.
__global__ void k_rowsum_fixed(const double* __restrict__ J, int N, const int32_t* __restrict__ fsite,
                               const double* __restrict__ fq, int Nf, double* __restrict__ s)
{
    int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= N) return;
    double acc = 0.0;
    for (int f = lane; f < Nf; f += 32) acc += J[(long)row * N + fsite[f]] * fq[f];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[row] = acc;
}

// phi_fix[v] = s[vsite[v]] (zero padded to ld); E_const = sum_f q_f s_f
// (one block of 256, fixed reduction order).
__global__ void k_fixed_finish(const double* __restrict__ s, const int32_t* __restrict__ vsite, int Nv, int ld,
                               const int32_t* __restrict__ fsite, const double* __restrict__ fq, int Nf,
                               double* __restrict__ phifix, double* __restrict__ E_const)
{
    for (int v = threadIdx.x; v < ld; v += blockDim.x) phifix[v] = v < Nv ? s[vsite[v]] : 0.0;
    __shared__ double red[256];
    double acc = 0.0;
    for (int f = threadIdx.x; f < Nf; f += blockDim.x) acc += fq[f] * s[fsite[f]];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E_const = red[0];
}

// ---------------------------------------------------------------------------
// Plain FP64 (and FP32) batched scoring: Phi = J_vv Q on CUDA cores, 64x64
// tiles, 4x4 outputs per thread, and the energy row-dot in the epilogue:
//   partial[mt][b] = sum_{i in tile mt} q_ib (Phi_ib + 2 phi_fix_i).
// ---------------------------------------------------------------------------
constexpr int PB_M = 64, PB_N = 64, PB_K = 16;

template <typename T, bool WANT_E, bool WANT_PHI>
__global__ void __launch_bounds__(256) k_phi(const T* __restrict__ Jvv, int ld, int Nv,
                                             const int8_t* __restrict__ species, int B, const double* __restrict__ z,
                                             const double* __restrict__ phifix, double* __restrict__ partial,
                                             T* __restrict__ phi_out)
{
    __shared__ T As[PB_K][PB_M + 1];
    __shared__ T Bs[PB_K][PB_N + 1];
    __shared__ double red[16][PB_N + 1];
    __shared__ double zs[64];
    const int b0 = blockIdx.x * PB_N, i0 = blockIdx.y * PB_M;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (threadIdx.x < 64) zs[threadIdx.x] = z[threadIdx.x < 64 ? threadIdx.x : 0];
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
    __syncthreads();
    for (int k0 = 0; k0 < Nv; k0 += PB_K) {
        for (int e = threadIdx.x; e < PB_M * PB_K; e += 256) {
            int r = e / PB_K, c = e % PB_K;
            int gi = i0 + r, gk = k0 + c;
            As[c][r] = Jvv[(long)gi * ld + gk];   // padded to ld >= multiple of 128, zero filled
            int gb = b0 + r;
            Bs[c][r] = (gb < B && gk < Nv) ? (T)zs[species[(long)gb * Nv + gk]] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PB_K; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ty * 4 + u];
                b[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    double colsum[4] = {0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int gi = i0 + ty * 4 + u;
        if (gi >= Nv) continue;
        double pf = phifix[gi];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gb = b0 + tx * 4 + v;
            if (gb >= B) continue;
            if (WANT_PHI) phi_out[(long)gb * Nv + gi] = (T)((double)acc[u][v] + pf);
            if (WANT_E) {
                double q = zs[species[(long)gb * Nv + gi]];
                colsum[v] += q * ((double)acc[u][v] + 2.0 * pf);
            }
        }
    }
    if (WANT_E) {
#pragma unroll
        for (int v = 0; v < 4; ++v) red[ty][tx * 4 + v] = colsum[v];
        __syncthreads();
        if (threadIdx.x < PB_N) {
            double s = 0.0;
            for (int r = 0; r < 16; ++r) s += red[r][threadIdx.x];
            int gb = b0 + threadIdx.x;
            if (gb < B) partial[(long)blockIdx.y * B + gb] = s;
        }
    }
}

__global__ void k_finish_E(const double* __restrict__ partial, int mtiles, int B, double E_const,
                           double* __restrict__ E)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
    for (int m = 0; m < mtiles; ++m) s += partial[(long)m * B + b];
    E[b] = s + E_const;
}

// Random valid structures: one thread per (configuration, class).
__global__ void k_random_configs(int B, int ncls, int S, const int32_t* __restrict__ cls_start,
                                 const int32_t* __restrict__ cls_pos, const int32_t* __restrict__ counts,
                                 uint64_t seed, int Nv, int8_t* __restrict__ out)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * ncls) return;
    int b = (int)(t / ncls), k = (int)(t % ncls);
    int8_t* o = out + (long)b * Nv;
    const int start = cls_start[k], n = cls_start[k + 1] - start;
    int f = 0;
    for (int s = 0; s < S; ++s)
        for (int r = 0; r < counts[k * S + s]; ++r) o[cls_pos[start + f++]] = (int8_t)s;
    uint4 blk = make_uint4(0, 0, 0, 0);
    for (int tt = 0; tt + 1 < n; ++tt) {
        int top = n - 1 - tt;
        if ((tt & 3) == 0) blk = goacd::philox_seed(seed, (uint32_t)(tt >> 2), (uint32_t)b, (uint32_t)k, 5u);
        uint32_t x = (tt & 3) == 0 ? blk.x : (tt & 3) == 1 ? blk.y : (tt & 3) == 2 ? blk.z : blk.w;
        int j = (int)goacd::draw_below(x, (uint32_t)(top + 1));
        int pa = cls_pos[start + top], pb = cls_pos[start + j];
        int8_t tmp = o[pa];
        o[pa] = o[pb];
        o[pb] = tmp;
    }
}

// FP64 rescoring of a few configurations over the upper block triangle of
// J_vv: block (I, J), I <= J, of 64 x 64 sites adds w sum_{i in I, j in J}
// q_bi J_ij q_bj for every configuration b (w = 1 on the diagonal, 2 above),
// configurations in chunks of 64, 4 threads per configuration.
constexpr int RS = 64;

__global__ void __launch_bounds__(256) k_rescore_pairs(const double* __restrict__ Jvv, int ld, int Nv,
                                                       const int8_t* __restrict__ sp, int k,
                                                       const double* __restrict__ z, double* __restrict__ partial)
{
    __shared__ double Jt[RS][RS + 1];
    __shared__ double qI[RS][RS + 1];
    __shared__ double qJ[RS][RS + 1];
    int t = blockIdx.x;
    int bj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
    while (bj * (bj + 1) / 2 > t) --bj;
    const int bi = t - bj * (bj + 1) / 2;   // bi <= bj
    const int i0 = bi * RS, j0 = bj * RS;
    const double w = bi == bj ? 1.0 : 2.0;
    for (int e = threadIdx.x; e < RS * RS; e += 256) {
        const int r = e / RS, c = e % RS;
        Jt[r][c] = Jvv[(long)(i0 + r) * ld + j0 + c];      // padded to ld, zeros beyond Nv
    }
    const int cfg = threadIdx.x >> 2, part = threadIdx.x & 3;
    for (int c0 = 0; c0 < k; c0 += RS) {
        __syncthreads();
        for (int e = threadIdx.x; e < RS * RS; e += 256) {
            const int c = e / RS, x = e % RS;
            const int b = c0 + c;
            qI[c][x] = (b < k && i0 + x < Nv) ? z[sp[(long)b * Nv + i0 + x]] : 0.0;
            qJ[c][x] = (b < k && j0 + x < Nv) ? z[sp[(long)b * Nv + j0 + x]] : 0.0;
        }
        __syncthreads();
        double acc = 0.0;
        for (int jj = part * 16; jj < part * 16 + 16; ++jj) {
            double tj = 0.0;
#pragma unroll 8
            for (int ii = 0; ii < RS; ++ii) tj = fma(qI[cfg][ii], Jt[ii][jj], tj);
            acc = fma(qJ[cfg][jj], tj, acc);
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (part == 0 && c0 + cfg < k) partial[(long)blockIdx.x * k + c0 + cfg] = w * acc;
    }
}

// E_b = E_const + 2 q_b . phi_fix + sum over block pairs (fixed order); one warp per configuration.
__global__ void k_rescore_finish(const double* __restrict__ partial, int npairs, int k, const int8_t* __restrict__ sp,
                                 int Nv, const double* __restrict__ z, const double* __restrict__ phifix,
                                 double E_const, double* __restrict__ E)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= k) return;
    double s = 0.0;
    for (int t = lane; t < npairs; t += 32) s += partial[(long)t * k + b];
    for (int v = lane; v < Nv; v += 32) s += z[sp[(long)b * Nv + v]] * (2.0 * phifix[v]);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) E[b] = s + E_const;
}

// rank of each E by (E, index) among B; entries with rank < k are selected.
__global__ void k_rank_select(const double* __restrict__ E, int B, int k, int* __restrict__ sel)
{
    __shared__ double tile[256];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ei = i < B ? E[i] : 0.0;
    int rank = 0;
    for (int j0 = 0; j0 < B; j0 += 256) {
        int j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < B ? E[j] : 0.0;
        __syncthreads();
        int lim = min(256, B - j0);
        if (i < B)
            for (int t = 0; t < lim; ++t) {
                double ej = tile[t];
                rank += (ej < ei) || (ej == ei && j0 + t < i);
            }
        __syncthreads();
    }
    if (i < B && rank < k) sel[rank] = i;
}

// Top-k selection in O(B) for large batches, with the result of k_rank_select
// (the k smallest (E, index)): E is mapped to an order-preserving 64-bit key
// (-0 read as +0), six passes of an 11-bit digit histogram over the keys that
// share the digits fixed so far find the key T of the k-th smallest, and an
// ordered compaction takes every key below T and the lowest-index keys equal
// to T.  The selected indices come out in index order (keys below T first).
constexpr int TK_BINS = 2048;
constexpr int TK_BLOCK = 1024;           // elements per compaction block: 256 threads x 4
constexpr int kTopkRankMax = 512;        // up to this batch the quadratic rank kernel is used

struct TopkState {
    unsigned long long prefix, mask;     // digits fixed so far and their bit mask
    int need, cnt_lt;                    // rank still wanted among keys matching prefix; keys below
};

__device__ __forceinline__ unsigned long long topk_key(double e)
{
    if (e == 0.0) e = 0.0;
    const unsigned long long u = (unsigned long long)__double_as_longlong(e);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_topk_init(TopkState* st, unsigned int* hist, int k)
{
    for (int i = threadIdx.x; i < TK_BINS; i += 256) hist[i] = 0u;
    if (threadIdx.x == 0) {
        st->prefix = 0ull;
        st->mask = 0ull;
        st->need = k;
        st->cnt_lt = 0;
    }
}

__global__ void __launch_bounds__(256) k_topk_hist(const double* __restrict__ E, int B, const TopkState* __restrict__ st,
                                                   int shift, unsigned int* __restrict__ hist)
{
    __shared__ unsigned int h[TK_BINS];
    for (int i = threadIdx.x; i < TK_BINS; i += 256) h[i] = 0u;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    for (long i = (long)blockIdx.x * 256 + threadIdx.x; i < B; i += (long)gridDim.x * 256) {
        const unsigned long long key = topk_key(E[i]);
        if (((key ^ prefix) & mask) == 0ull) atomicAdd(&h[(key >> shift) & (TK_BINS - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TK_BINS; i += 256)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One block: the bin holding rank `need` among the counted keys fixes the next digit.
__global__ void __launch_bounds__(256) k_topk_pick(TopkState* st, unsigned int* hist, int shift)
{
    __shared__ unsigned int part[256];
    __shared__ int found_v;
    __shared__ unsigned int found_below;
    const int t = threadIdx.x;
    const unsigned int need = (unsigned int)st->need;
    unsigned int loc[TK_BINS / 256], sum = 0u;
#pragma unroll
    for (int u = 0; u < TK_BINS / 256; ++u) {
        loc[u] = hist[t * (TK_BINS / 256) + u];
        sum += loc[u];
    }
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {             // inclusive scan over the 256 partial sums
        const unsigned int v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const unsigned int excl = part[t] - sum;
    if (excl < need && need <= part[t]) {           // exactly one thread
        unsigned int c = excl;
#pragma unroll
        for (int u = 0; u < TK_BINS / 256; ++u) {
            if (c + loc[u] >= need) {
                found_v = t * (TK_BINS / 256) + u;
                found_below = c;
                break;
            }
            c += loc[u];
        }
    }
#pragma unroll
    for (int u = 0; u < TK_BINS / 256; ++u) hist[t * (TK_BINS / 256) + u] = 0u;
    __syncthreads();
    if (t == 0) {
        st->prefix |= (unsigned long long)found_v << shift;
        st->mask |= (unsigned long long)(TK_BINS - 1) << shift;
        st->need -= (int)found_below;
        st->cnt_lt += (int)found_below;
    }
}

// Per 1024-element block: keys below T and keys equal to T.
__global__ void __launch_bounds__(256) k_topk_count(const double* __restrict__ E, int B, const TopkState* __restrict__ st,
                                                    int2* __restrict__ cnt)
{
    __shared__ int red[2][8];
    const unsigned long long T = st->prefix;
    const long base = (long)blockIdx.x * TK_BLOCK;
    int lt = 0, eq = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long i = base + threadIdx.x * 4 + u;
        if (i < B) {
            const unsigned long long key = topk_key(E[i]);
            lt += key < T;
            eq += key == T;
        }
    }
    lt = __reduce_add_sync(0xffffffffu, lt);
    eq = __reduce_add_sync(0xffffffffu, eq);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = lt;
        red[1][threadIdx.x >> 5] = eq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < 8; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        cnt[blockIdx.x] = make_int2(a, b);
    }
}

// One block: exclusive scan of the per-block counts, in block order.
__global__ void __launch_bounds__(1024) k_topk_scan(const int2* __restrict__ cnt, int nb, int2* __restrict__ off)
{
    __shared__ int wl[32], we[32];
    __shared__ int carry_l, carry_e;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_l = carry_e = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const int2 v = b < nb ? cnt[b] : make_int2(0, 0);
        int l = v.x, e = v.y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int tl = __shfl_up_sync(0xffffffffu, l, o), te = __shfl_up_sync(0xffffffffu, e, o);
            if (lane >= o) {
                l += tl;
                e += te;
            }
        }
        if (lane == 31) {
            wl[wid] = l;
            we[wid] = e;
        }
        __syncthreads();
        if (wid == 0) {
            int xl = wl[lane], xe = we[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tl = __shfl_up_sync(0xffffffffu, xl, o), te = __shfl_up_sync(0xffffffffu, xe, o);
                if (lane >= o) {
                    xl += tl;
                    xe += te;
                }
            }
            wl[lane] = xl;
            we[lane] = xe;
        }
        __syncthreads();
        const int pl = carry_l + (wid ? wl[wid - 1] : 0), pe = carry_e + (wid ? we[wid - 1] : 0);
        if (b < nb) off[b] = make_int2(pl + l - v.x, pe + e - v.y);
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_l += wl[31];
            carry_e += we[31];
        }
        __syncthreads();
    }
}

// Per 1024-element block: keys below T to sel[off.x ...], keys equal to T to
// sel[cnt_lt + off.y ...] while fewer than `need` have been placed; index order.
__global__ void __launch_bounds__(256) k_topk_write(const double* __restrict__ E, int B, const TopkState* __restrict__ st,
                                                    const int2* __restrict__ off, int* __restrict__ sel)
{
    __shared__ int wl[8], we[8];
    const unsigned long long T = st->prefix;
    const int need = st->need, cnt_lt = st->cnt_lt;
    const int2 o = off[blockIdx.x];
    if (o.x >= cnt_lt && o.y >= need) return;       // nothing of this block is selected (uniform)
    const long base = (long)blockIdx.x * TK_BLOCK;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool fl[4], fe[4];
    int nl = 0, ne = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long i = base + threadIdx.x * 4 + u;
        fl[u] = fe[u] = false;
        if (i < B) {
            const unsigned long long key = topk_key(E[i]);
            fl[u] = key < T;
            fe[u] = key == T;
        }
        nl += fl[u];
        ne += fe[u];
    }
    int il = nl, ie = ne;                            // inclusive scans in thread order
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int tl = __shfl_up_sync(0xffffffffu, il, d), te = __shfl_up_sync(0xffffffffu, ie, d);
        if (lane >= d) {
            il += tl;
            ie += te;
        }
    }
    if (lane == 31) {
        wl[wid] = il;
        we[wid] = ie;
    }
    __syncthreads();
    int pl = 0, pe = 0;
    for (int w = 0; w < wid; ++w) {
        pl += wl[w];
        pe += we[w];
    }
    int rl = o.x + pl + il - nl, re = o.y + pe + ie - ne;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = (int)(base + threadIdx.x * 4 + u);
        if (fl[u]) sel[rl++] = i;
        if (fe[u]) {
            if (re < need) sel[cnt_lt + re] = i;
            ++re;
        }
    }
}

__global__ void k_gather_rows(const int8_t* __restrict__ src, int Nv, const int* __restrict__ sel, int k,
                              int8_t* __restrict__ dst)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)k * Nv) return;
    int r = (int)(t / Nv), c = (int)(t % Nv);
    dst[t] = src[(long)sel[r] * Nv + c];
}

// sort k (<= 1024) rescored entries by (E64, original index); one block.
__global__ void k_sort_small(const double* __restrict__ E64, const int* __restrict__ sel, int k,
                             int* __restrict__ idx_out, double* __restrict__ E_out)
{
    __shared__ double e[1024];
    __shared__ int id[1024];
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        e[t] = E64[t];
        id[t] = sel[t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        int r = 0;
        for (int u = 0; u < k; ++u) r += (e[u] < e[t]) || (e[u] == e[t] && id[u] < id[t]);
        idx_out[r] = id[t];
        E_out[r] = e[t];
    }
}

}  // namespace

namespace goac {

template <typename T>
static goac_status score_cuda_core(goac_problem* p, const T* J, const int8_t* species, int B, double* E_out,
                                   T* phi_out)
{
    goac_ctx* ctx = p->ctx;
    const int mt = (p->Nv + PB_M - 1) / PB_M;
    dim3 grid((B + PB_N - 1) / PB_N, mt);
    if (E_out) {
        goac_status rc = ensure(p->partial, sizeof(double) * (size_t)mt * B);
        if (rc) return rc;
    }
    double* part = (double*)p->partial.ptr;
    KTimer kt(ctx, KID_SCORE_CC, ctx->stream);
    if (E_out && phi_out)
        goac::launch(k_phi<T, true, true>, grid, 256, 0, ctx->stream, J, p->Nv_pad, p->Nv, species, B, p->z_dev, p->phifix,
                                                            part, phi_out);
    else if (E_out)
        goac::launch(k_phi<T, true, false>, grid, 256, 0, ctx->stream, J, p->Nv_pad, p->Nv, species, B, p->z_dev, p->phifix,
                                                             part, nullptr);
    else
        goac::launch(k_phi<T, false, true>, grid, 256, 0, ctx->stream, J, p->Nv_pad, p->Nv, species, B, p->z_dev, p->phifix,
                                                             nullptr, phi_out);
    GOAC_LAUNCH_CHECK("k_phi");
    if (E_out) {
        goac::launch(k_finish_E, (B + 255) / 256, 256, 0, ctx->stream, part, mt, B, p->E_const, E_out);
        GOAC_LAUNCH_CHECK("k_finish_E");
    }
    return GOAC_OK;
}

goac_status score_f64(goac_problem* p, const int8_t* species, int B, double* E_out, double* phi_out)
{
    return score_cuda_core<double>(p, p->J_vv, species, B, E_out, phi_out);
}

goac_status score_f32(goac_problem* p, const int8_t* species, int B, double* E_out, float* phi_out)
{
    goac_status rc = prepare_f32(p);
    if (rc) return rc;
    return score_cuda_core<float>(p, p->J_f32, species, B, E_out, phi_out);
}

}  // namespace goac

// ---------------------------------------------------------------------------
// Problem API
// ---------------------------------------------------------------------------
extern "C" goac_status goac_problem_create(goac_ctx* ctx, const double* J_dev, int32_t N,
                                           const int32_t* site_class_host, const double* fixed_q_host,
                                           const double* z_host, int32_t S, const int32_t* counts_host,
                                           int32_t n_class, int32_t allow_charged, goac_problem** out)
{
    if (!ctx || !J_dev || !site_class_host || !fixed_q_host || !z_host || !counts_host || !out)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: null pointer");
    *out = nullptr;
    if (N <= 0 || S <= 0 || S > 64 || n_class <= 0)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: need N > 0, 0 < S <= 64, n_class > 0");
    std::vector<int32_t> vsite, fsite;
    std::vector<double> fq;
    std::vector<int32_t> csize(n_class, 0);
    for (int i = 0; i < N; ++i) {
        int c = site_class_host[i];
        if (c < -1 || c >= n_class) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: bad site class");
        if (c < 0) {
            fsite.push_back(i);
            fq.push_back(fixed_q_host[i]);
        } else {
            vsite.push_back(i);
            csize[c]++;
        }
    }
    const int Nv = (int)vsite.size();
    if (Nv == 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: no variable sites");
    double qtot = 0.0;
    for (double q : fq) qtot += q;
    for (int k = 0; k < n_class; ++k) {
        long sum = 0;
        for (int s = 0; s < S; ++s) {
            if (counts_host[k * S + s] < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: negative count");
            sum += counts_host[k * S + s];
            qtot += counts_host[k * S + s] * z_host[s];
        }
        if (sum != csize[k])
            return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: counts of class " + std::to_string(k) +
                                                        " do not add up to its " + std::to_string(csize[k]) +
                                                        " positions");
    }
    if (!allow_charged && fabs(qtot) > 1e-9)
        return goac::fail(GOAC_ERR_NOT_NEUTRAL, "goac_problem_create: total charge " + std::to_string(qtot) +
                                                    " is not neutral");
    GOAC_CUDA(cudaSetDevice(ctx->device));

    goac_problem* p = new goac_problem();
    p->ctx = ctx;
    p->N = N;
    p->Nv = Nv;
    p->S = S;
    p->ncls = n_class;
    p->Nv_pad = ((Nv + 127) / 128) * 128;
    p->has_fixed = !fsite.empty();
    p->z.assign(z_host, z_host + S);
    p->counts.assign(counts_host, counts_host + n_class * S);
    p->vclass.resize(Nv);
    for (int v = 0; v < Nv; ++v) p->vclass[v] = site_class_host[vsite[v]];
    p->cls_start.assign(n_class + 1, 0);
    for (int v = 0; v < Nv; ++v) p->cls_start[p->vclass[v] + 1]++;
    for (int k = 0; k < n_class; ++k) p->cls_start[k + 1] += p->cls_start[k];
    p->cls_pos.resize(Nv);
    {
        std::vector<int32_t> fill(n_class, 0);
        for (int v = 0; v < Nv; ++v) {
            int k = p->vclass[v];
            p->cls_pos[p->cls_start[k] + fill[k]++] = v;
        }
    }
    std::vector<int32_t> cls_rank(Nv);
    for (int q = 0; q < Nv; ++q) cls_rank[p->cls_pos[q]] = q;
    p->wprefix.resize(n_class);
    uint64_t acc = 0;
    for (int k = 0; k < n_class; ++k) {
        uint64_t n = (uint64_t)(p->cls_start[k + 1] - p->cls_start[k]);
        if (n >= 2) {
            p->nmovable++;
            p->only_movable = k;
            acc += n * (n - 1);
        }
        p->wprefix[k] = (uint32_t)acc;
    }
    if (acc >= (1ull << 32)) {
        delete p;
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_create: class too large");
    }
    p->wtotal = (uint32_t)acc;

    const int ld = p->Nv_pad;
    const int Nf = (int)fsite.size();
    int32_t *d_vsite = nullptr, *d_fsite = nullptr;
    double *d_fq = nullptr, *d_s = nullptr, *d_ec = nullptr;
    goac_status rc = GOAC_OK;
#define PTRY(call)                                        \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess && rc == GOAC_OK) rc = goac::cuda_fail(e__, #call); \
    } while (0)
    PTRY(cudaMalloc(&p->J_vv, sizeof(double) * (size_t)ld * ld));
    PTRY(cudaMalloc(&p->diag, sizeof(double) * Nv));
    PTRY(cudaMalloc(&p->phifix, sizeof(double) * ld));
    PTRY(cudaMalloc(&p->z_dev, sizeof(double) * 64));
    PTRY(cudaMalloc(&p->vclass_dev, sizeof(int32_t) * Nv));
    PTRY(cudaMalloc(&p->cls_start_dev, sizeof(int32_t) * (n_class + 1)));
    PTRY(cudaMalloc(&p->cls_pos_dev, sizeof(int32_t) * Nv));
    PTRY(cudaMalloc(&p->cls_rank_dev, sizeof(int32_t) * Nv));
    PTRY(cudaMalloc(&p->counts_dev, sizeof(int32_t) * n_class * S));
    PTRY(cudaMalloc(&p->wprefix_dev, sizeof(uint32_t) * n_class));
    PTRY(cudaMalloc(&d_vsite, sizeof(int32_t) * Nv));
    PTRY(cudaMalloc(&d_fsite, sizeof(int32_t) * (Nf + 1)));
    PTRY(cudaMalloc(&d_fq, sizeof(double) * (Nf + 1)));
    PTRY(cudaMalloc(&d_s, sizeof(double) * N));
    PTRY(cudaMalloc(&d_ec, sizeof(double)));
    if (rc == GOAC_OK) {
        cudaStream_t st = ctx->stream;
        std::vector<double> z64(64, 0.0);
        for (int s = 0; s < S; ++s) z64[s] = z_host[s];
        PTRY(cudaMemcpyAsync(p->z_dev, z64.data(), sizeof(double) * 64, cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->vclass_dev, p->vclass.data(), sizeof(int32_t) * Nv, cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->cls_start_dev, p->cls_start.data(), sizeof(int32_t) * (n_class + 1),
                             cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->cls_pos_dev, p->cls_pos.data(), sizeof(int32_t) * Nv, cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->cls_rank_dev, cls_rank.data(), sizeof(int32_t) * Nv, cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->counts_dev, counts_host, sizeof(int32_t) * n_class * S, cudaMemcpyHostToDevice, st));
        PTRY(cudaMemcpyAsync(p->wprefix_dev, p->wprefix.data(), sizeof(uint32_t) * n_class, cudaMemcpyHostToDevice,
                             st));
        PTRY(cudaMemcpyAsync(d_vsite, vsite.data(), sizeof(int32_t) * Nv, cudaMemcpyHostToDevice, st));
        if (Nf) {
            PTRY(cudaMemcpyAsync(d_fsite, fsite.data(), sizeof(int32_t) * Nf, cudaMemcpyHostToDevice, st));
            PTRY(cudaMemcpyAsync(d_fq, fq.data(), sizeof(double) * Nf, cudaMemcpyHostToDevice, st));
        }
        if (rc == GOAC_OK) {
            long total = (long)ld * ld;
            int blocks = (int)std::min<long>((total + 255) / 256, 65535L * 8);
            goac::launch(k_gather_jvv, blocks, 256, 0, st, J_dev, N, d_vsite, Nv, ld, p->J_vv, p->diag);
            goac::launch(k_rowsum_fixed, (N + 7) / 8, 256, 0, st, J_dev, N, d_fsite, d_fq, Nf, d_s);
            goac::launch(k_fixed_finish, 1, 256, 0, st, d_s, d_vsite, Nv, ld, d_fsite, d_fq, Nf, p->phifix, d_ec);
            PTRY(cudaGetLastError());
            PTRY(cudaMemcpyAsync(&p->E_const, d_ec, sizeof(double), cudaMemcpyDeviceToHost, st));
            PTRY(cudaStreamSynchronize(st));
        }
    }
#undef PTRY
    cudaFree(d_vsite);
    cudaFree(d_fsite);
    cudaFree(d_fq);
    cudaFree(d_s);
    cudaFree(d_ec);
    if (rc != GOAC_OK) {
        goac_problem_destroy(p);
        return rc;
    }
    *out = p;
    return GOAC_OK;
}

extern "C" goac_status goac_problem_destroy(goac_problem* p)
{
    if (!p) return GOAC_OK;
    if (p->ctx) {
        cudaSetDevice(p->ctx->device);
        cudaStreamSynchronize(p->ctx->stream);
    }
    cudaFree(p->J_vv);
    cudaFree(p->diag);
    cudaFree(p->phifix);
    cudaFree(p->z_dev);
    cudaFree(p->vclass_dev);
    cudaFree(p->cls_start_dev);
    cudaFree(p->cls_pos_dev);
    cudaFree(p->cls_rank_dev);
    cudaFree(p->counts_dev);
    cudaFree(p->wprefix_dev);
    cudaFree(p->J_bf16);
    cudaFree(p->J_tf32);
    cudaFree(p->J_tf32_full);
    cudaFree(p->J_f16_full);
    cudaFree(p->phifix_f32);
    cudaFree(p->f16_exp);
    cudaFree(p->J_f32);
    cudaFree(p->diag_f32);
    free_buf(p->qt);
    free_buf(p->qi);
    free_buf(p->partial);
    free_buf(p->phi);
    free_buf(p->score_tmp);
    free_buf(p->topk_tmp);
    free_buf(p->grad_tmp);
    free_buf(p->ga_incr);
    free_buf(p->ga_buf);
    free_buf(p->ga_dev);
    free_buf(p->sched.buf);
    free_buf(p->sched_ex.buf);
    cudaFree(p->J_dig);
    cudaFree(p->dig_exp);
    cudaFree(p->zq_dev);
    cudaFree(p->J_dig_full);
    cudaFree(p->dig_exp_full);
    free_buf(p->phi_dig);
    delete p;
    return GOAC_OK;
}

extern "C" goac_status goac_problem_info(const goac_problem* p, int32_t* Nv, double* E_const)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_info: NULL problem");
    if (Nv) *Nv = p->Nv;
    if (E_const) *E_const = p->E_const;
    return GOAC_OK;
}

extern "C" goac_status goac_problem_phi_fix(const goac_problem* p, double* phi_fix_dev)
{
    if (!p || !phi_fix_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_phi_fix: NULL argument");
    GOAC_CUDA(cudaMemcpyAsync(phi_fix_dev, p->phifix, sizeof(double) * p->Nv, cudaMemcpyDeviceToDevice,
                              p->ctx->stream));
    return GOAC_OK;
}

extern "C" goac_status goac_problem_exact_info(const goac_problem* p, int32_t* digit_bits, int32_t* digits,
                                               int32_t* charge_shift)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_problem_exact_info: NULL problem");
    return goac::exact_info(p, digit_bits, digits, charge_shift);
}

extern "C" goac_status goac_score(goac_problem* p, const int8_t* species_dev, int32_t B, int32_t precision,
                                  double* E_dev)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score: NULL problem");
    if (B <= 0 || B > GOAC_MAX_BATCH)
        return B == 0 ? GOAC_OK : goac::fail(GOAC_ERR_INVALID_ARG, "goac_score: B < 0 or B > GOAC_MAX_BATCH");
    if (!species_dev || !E_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    switch (precision) {
        case GOAC_PREC_F64: return goac::score_f64(p, species_dev, B, E_dev, nullptr);
        case GOAC_PREC_F32: return goac::score_f32(p, species_dev, B, E_dev, nullptr);
        case GOAC_PREC_TF32:
        case GOAC_PREC_TF32X2:
        case GOAC_PREC_BF16X2:
        case GOAC_PREC_BF16X3:
        case GOAC_PREC_EXACT: return goac::score_tc(p, species_dev, B, precision, E_dev);
        default: return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score: unknown precision");
    }
}

extern "C" goac_status goac_score_host(goac_problem* p, const int8_t* species_host, int32_t B, int32_t precision,
                                       double* E_host)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host: NULL problem");
    if (B <= 0 || B > GOAC_MAX_BATCH)
        return B == 0 ? GOAC_OK : goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host: B < 0 or B > GOAC_MAX_BATCH");
    if (!species_host || !E_host) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host: NULL argument");
    goac_ctx* ctx = p->ctx;
    GOAC_CUDA(cudaSetDevice(ctx->device));
    size_t sb = (size_t)B * p->Nv, eb = sizeof(double) * (size_t)B;
    goac_status rc = goac::ensure(ctx->host_io_species, sb);
    if (!rc) rc = goac::ensure(ctx->host_io_E, eb);
    if (rc) return rc;
    GOAC_CUDA(cudaMemcpyAsync(ctx->host_io_species.ptr, species_host, sb, cudaMemcpyHostToDevice, ctx->stream));
    rc = goac_score(p, (const int8_t*)ctx->host_io_species.ptr, B, precision, (double*)ctx->host_io_E.ptr);
    if (rc) return rc;
    GOAC_CUDA(cudaMemcpyAsync(E_host, ctx->host_io_E.ptr, eb, cudaMemcpyDeviceToHost, ctx->stream));
    GOAC_CUDA(cudaStreamSynchronize(ctx->stream));
    return GOAC_OK;
}

extern "C" goac_status goac_score_host_async(goac_problem* p, const int8_t* species_host, int32_t B,
                                             int32_t precision, double* E_host)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host_async: NULL problem");
    if (B <= 0 || B > GOAC_MAX_BATCH)
        return B == 0 ? GOAC_OK : goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host_async: B < 0 or B > GOAC_MAX_BATCH");
    if (!species_host || !E_host) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_host_async: NULL argument");
    goac_ctx* ctx = p->ctx;
    GOAC_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->copy_stream) {
        GOAC_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (int s = 0; s < 2; ++s) {
            GOAC_CUDA(cudaEventCreateWithFlags(&ctx->async_h2d[s], cudaEventDisableTiming));
            GOAC_CUDA(cudaEventCreateWithFlags(&ctx->async_done[s], cudaEventDisableTiming));
        }
    }
    const int s = ctx->async_next;
    const size_t sb = (size_t)B * p->Nv, eb = sizeof(double) * (size_t)B;
    if (ctx->async_species[s].bytes < sb || ctx->async_E[s].bytes < eb) {
        // growing a slot frees its old buffer: let the work that uses it finish first
        if (ctx->async_used[s]) GOAC_CUDA(cudaEventSynchronize(ctx->async_done[s]));
        goac_status rc = goac::ensure(ctx->async_species[s], sb);
        if (!rc) rc = goac::ensure(ctx->async_E[s], eb);
        if (rc) return rc;
    }
    if (ctx->async_used[s]) GOAC_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->async_done[s], 0));
    GOAC_CUDA(cudaMemcpyAsync(ctx->async_species[s].ptr, species_host, sb, cudaMemcpyHostToDevice, ctx->copy_stream));
    GOAC_CUDA(cudaEventRecord(ctx->async_h2d[s], ctx->copy_stream));
    GOAC_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->async_h2d[s], 0));
    goac_status rc = goac_score(p, (const int8_t*)ctx->async_species[s].ptr, B, precision, (double*)ctx->async_E[s].ptr);
    if (rc) return rc;
    GOAC_CUDA(cudaMemcpyAsync(E_host, ctx->async_E[s].ptr, eb, cudaMemcpyDeviceToHost, ctx->stream));
    GOAC_CUDA(cudaEventRecord(ctx->async_done[s], ctx->stream));
    ctx->async_used[s] = true;
    ctx->async_next = s ^ 1;
    return GOAC_OK;
}

extern "C" goac_status goac_topk_rescore(goac_problem* p, const int8_t* species_dev, int32_t B,
                                         const double* E_approx_dev, int32_t k, int32_t* idx_dev, double* E_dev)
{
    if (!p || !species_dev || !E_approx_dev || !idx_dev || !E_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_topk_rescore: NULL argument");
    if (k < 1 || k > 1024 || k > B || B > GOAC_MAX_BATCH) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_topk_rescore: need 1 <= k <= min(B, 1024)");
    goac_ctx* ctx = p->ctx;
    GOAC_CUDA(cudaSetDevice(ctx->device));
    const int nb = (p->Nv + RS - 1) / RS;
    const long npairs = (long)nb * (nb + 1) / 2;
    const int nblk = (int)(((long)B + TK_BLOCK - 1) / TK_BLOCK);
    const size_t sub_bytes = ((size_t)k * p->Nv + 255) & ~(size_t)255;
    size_t need = sizeof(int) * 1024 + sizeof(double) * 1024 + sizeof(double) * (size_t)npairs * k + sub_bytes;
    const size_t radix_at = need;
    if (B > kTopkRankMax) need += 256 + sizeof(unsigned int) * TK_BINS + 2 * sizeof(int2) * (size_t)nblk;
    goac_status rc = goac::ensure(p->topk_tmp, need);
    if (rc) return rc;
    int* sel = (int*)p->topk_tmp.ptr;
    double* e64 = (double*)((char*)p->topk_tmp.ptr + sizeof(int) * 1024);
    double* part = e64 + 1024;
    int8_t* sub = (int8_t*)(part + (size_t)npairs * k);
    if (B <= kTopkRankMax) {
        goac::launch(k_rank_select, (B + 255) / 256, 256, 0, ctx->stream, E_approx_dev, B, k, sel);
    } else {
        TopkState* st = (TopkState*)((char*)p->topk_tmp.ptr + radix_at);
        unsigned int* hist = (unsigned int*)((char*)st + 256);
        int2* cnt = (int2*)(hist + TK_BINS);
        int2* off = cnt + nblk;
        goac::launch(k_topk_init, 1, 256, 0, ctx->stream, st, hist, k);
        const int hgrid = (int)std::min<long>(((long)B + 255) / 256, (long)ctx->num_sms * 8);
        const int shifts[6] = {53, 42, 31, 20, 9, 0};
        for (int ps = 0; ps < 6; ++ps) {
            goac::launch(k_topk_hist, hgrid, 256, 0, ctx->stream, E_approx_dev, B, (const TopkState*)st, shifts[ps],
                         hist);
            goac::launch(k_topk_pick, 1, 256, 0, ctx->stream, st, hist, shifts[ps]);
        }
        goac::launch(k_topk_count, nblk, 256, 0, ctx->stream, E_approx_dev, B, (const TopkState*)st, cnt);
        goac::launch(k_topk_scan, 1, 1024, 0, ctx->stream, (const int2*)cnt, nblk, off);
        goac::launch(k_topk_write, nblk, 256, 0, ctx->stream, E_approx_dev, B, (const TopkState*)st,
                     (const int2*)off, sel);
    }
    goac::launch(k_gather_rows, (int)(((long)k * p->Nv + 255) / 256), 256, 0, ctx->stream, species_dev, p->Nv, sel, k, sub);
    GOAC_LAUNCH_CHECK("topk select");
    goac::launch(k_rescore_pairs, (unsigned)npairs, 256, 0, ctx->stream, (const double*)p->J_vv, p->Nv_pad, p->Nv,
                 (const int8_t*)sub, k, (const double*)p->z_dev, part);
    GOAC_LAUNCH_CHECK("k_rescore_pairs");
    goac::launch(k_rescore_finish, (k + 7) / 8, 256, 0, ctx->stream, (const double*)part, (int)npairs, k,
                 (const int8_t*)sub, p->Nv, (const double*)p->z_dev, (const double*)p->phifix, p->E_const, e64);
    GOAC_LAUNCH_CHECK("k_rescore_finish");
    goac::launch(k_sort_small, 1, 1024, 0, ctx->stream, e64, sel, k, idx_dev, E_dev);
    GOAC_LAUNCH_CHECK("k_sort_small");
    return GOAC_OK;
}

extern "C" goac_status goac_random_configs(goac_problem* p, int32_t B, uint64_t seed, int8_t* species_dev)
{
    if (!p || B < 0 || B > GOAC_MAX_BATCH) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_random_configs: bad argument");
    if (B == 0) return GOAC_OK;
    if (!species_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_random_configs: NULL output");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    long t = (long)B * p->ncls;
    goac::launch(k_random_configs, (int)((t + 127) / 128), 128, 0, p->ctx->stream, B, p->ncls, p->S, p->cls_start_dev,
                                                                         p->cls_pos_dev, p->counts_dev, seed, p->Nv,
                                                                         species_dev);
    GOAC_LAUNCH_CHECK("k_random_configs");
    return GOAC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free FP64 scoring.
//
// For callers that may not allocate device memory themselves: code whose
// device memory all comes from a host framework's own pool, or that runs under
// a policy of no allocation after start-up.  They pass every input and output
// buffer; the only other memory this entry point uses is the file-scope array
// below, which holds the per-tile partial energies of the FP64 scoring kernel.
// The array exists on every GPU that loads this library, for the life of the
// process.  It is shared by all calls on a device and keeps the last call's
// contents; the kernel writes every entry it later reads, so nothing needs
// clearing.  Calls whose work overlaps on the GPU race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr long kStaticPartialEntries = 1L << 19;   // 524,288 doubles = 4 MiB

__device__ __align__(256) double g_static_partial[kStaticPartialEntries];

std::mutex g_static_mu;
double* g_static_ptr[64] = {};   // device address of g_static_partial per device ordinal

}  // namespace

extern "C" goac_status goac_score_f64_noalloc(const double* Jvv_dev, int32_t ld, int32_t Nv,
                                              const int8_t* species_dev, int32_t B, const double* z_dev,
                                              const double* phi_fix_dev, double E_const, void* stream,
                                              double* E_dev)
{
    if (!Jvv_dev || !z_dev || !phi_fix_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_f64_noalloc: NULL argument");
    if (Nv <= 0 || B < 0 || B > GOAC_MAX_BATCH)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_f64_noalloc: need Nv > 0, 0 <= B <= GOAC_MAX_BATCH");
    const long mt = (Nv + PB_M - 1) / PB_M;
    if (ld < mt * PB_M)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_f64_noalloc: ld must be >= Nv rounded up to 64");
    if (B == 0) return GOAC_OK;
    if (!species_dev || !E_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_f64_noalloc: NULL argument");
    if (mt * (long)B > kStaticPartialEntries)
        return goac::fail(GOAC_ERR_INVALID_ARG,
                          "goac_score_f64_noalloc: ceil(Nv/64) * B = " + std::to_string(mt * (long)B) +
                              " exceeds the fixed scratch of 524288 entries");
    int dev = 0;
    GOAC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_score_f64_noalloc: device ordinal >= 64");
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GOAC_CUDA(cudaStreamIsCapturing(st, &cap));
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            // outside a stream capture the address is looked up on every call, so a device whose
            // context was reset (and the library's module loaded again) gets the array's new address
            void* p = nullptr;
            GOAC_CUDA(cudaGetSymbolAddress(&p, g_static_partial));
            g_static_ptr[dev] = (double*)p;
        } else if (!g_static_ptr[dev]) {
            return goac::fail(GOAC_ERR_INVALID_ARG,
                              "goac_score_f64_noalloc: the first call on a device must come before any stream capture");
        }
        part = g_static_ptr[dev];
    }
    dim3 grid((B + PB_N - 1) / PB_N, (unsigned)mt);
    goac::launch(k_phi<double, true, false>, grid, 256, 0, st, Jvv_dev, ld, Nv, species_dev, B, z_dev, phi_fix_dev,
                 part, (double*)nullptr);
    GOAC_LAUNCH_CHECK("k_phi (no-alloc)");
    goac::launch(k_finish_E, (B + 255) / 256, 256, 0, st, (const double*)part, (int)mt, B, E_const, E_dev);
    GOAC_LAUNCH_CHECK("k_finish_E (no-alloc)");
    return GOAC_OK;
}

// ---------------------------------------------------------------------------
// Failure-detection self test: one thread waits on an mbarrier that nothing
// arrives on, with the same clock-bounded wait the tensor-core kernels use.
// The wait runs out, the kernel records GOAC_ERR_TIMEOUT in the device error
// word and returns; the context stays usable.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_selftest_wait(long long limit_cycles, int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    goacd::mbar_init(&bar, 1);
    goacd::fence_barrier_init();
    if (!goacd::mbar_wait_bounded(&bar, 0, limit_cycles)) goacd::report(err, GOAC_ERR_TIMEOUT, 99, 0);
}

}  // namespace

extern "C" goac_status goac_selftest_wait_timeout(goac_ctx* ctx, int64_t limit_cycles)
{
    if (!ctx || limit_cycles <= 0 || limit_cycles > 4000000000LL)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_selftest_wait_timeout: bad argument");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    goac::launch(k_selftest_wait, 1, 32, 0, ctx->stream, (long long)limit_cycles, ctx->d_err);
    GOAC_LAUNCH_CHECK("k_selftest_wait");
    return goac::check_device_error(ctx);
}
