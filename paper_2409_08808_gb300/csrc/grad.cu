// Relaxed occupations and their hand-written adjoint, and rounding back to
// valid integer configurations.  (The paper's gradient descent is discrete,
// SI Gradient Descent; the relaxed form seeds MC / GA populations.)
//
//   p_vs = softmax over the species allowed in v's class of the logits L_vs
//   q_v  = sum_s p_vs z_s                      (fixed sites keep their charge)
//   E    = q^T J q + lambda sum_{k,s allowed} (sum_{v in k} p_vs - n_ks)^2
//   g_vs = z_s (2 J q)_v + 2 lambda (sum_{w in k} p_ws - n_ks)
//   dE/dL_vs = p_vs (g_vs - sum_t p_vt g_vt)
//
// (2 J q)_v = 2 (J_vv q_v + phi_fix)_v.  Two paths: the FP64 check path (FP64
// softmax, tiled FP64 GEMM on the CUDA cores, FP64 chain rule), and the fast
// path, where one FP32 pass forms p, q and q's TF32 hi / lo planes, the
// contraction runs on the tcgen05 tensor cores with both J and Q split into
// TF32 hi / lo (three products), and the chain rule runs in FP32 with the
// energy accumulated in FP64.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

__global__ void k_softmax(const float* __restrict__ logits, long BN, int Nv, int S, const int32_t* __restrict__ vclass,
                          const int32_t* __restrict__ counts, const double* __restrict__ z, double* __restrict__ p,
                          double* __restrict__ q)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= BN) return;
    const int v = (int)(t % Nv);
    const int k = vclass[v];
    const float* L = logits + t * S;
    double m = -INFINITY;
    for (int s = 0; s < S; ++s)
        if (counts[k * S + s] > 0 && (double)L[s] > m) m = (double)L[s];
    double den = 0.0;
    for (int s = 0; s < S; ++s) {
        const double e = counts[k * S + s] > 0 ? exp((double)L[s] - m) : 0.0;
        p[t * S + s] = e;
        den += e;
    }
    double qv = 0.0;
    for (int s = 0; s < S; ++s) {
        const double ps = p[t * S + s] / den;
        p[t * S + s] = ps;
        qv += ps * z[s];
    }
    q[t] = qv;
}

// colsum[(b*ncls + k)*S + s] = sum_{v in class k} p[b][v][s]; one block per (b, k).
__global__ void k_colsum(const double* __restrict__ p, int Nv, int S, int ncls, const int32_t* __restrict__ cls_start,
                         const int32_t* __restrict__ cls_pos, double* __restrict__ colsum)
{
    __shared__ double red[256];
    const int b = blockIdx.x / ncls, k = blockIdx.x % ncls;
    const int cs = cls_start[k], ce = cls_start[k + 1];
    for (int s = 0; s < S; ++s) {
        double acc = 0.0;
        for (int i = cs + threadIdx.x; i < ce; i += blockDim.x) acc += p[((long)b * Nv + cls_pos[i]) * S + s];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) colsum[((long)b * ncls + k) * S + s] = red[0];
        __syncthreads();
    }
}

// Phi[b][v] = sum_w J_vv[v][w] Q[b][w] (FP64, 64x64 tiles, 4x4 per thread).
constexpr int GM = 64, GK = 16;

__global__ void __launch_bounds__(256) k_phi_real(const double* __restrict__ J, int ld, int Nv,
                                                  const double* __restrict__ Q, int B, double* __restrict__ Phi)
{
    __shared__ double As[GK][GM + 1];
    __shared__ double Bs[GK][GM + 1];
    const int b0 = blockIdx.x * GM, i0 = blockIdx.y * GM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < Nv; k0 += GK) {
        for (int e = threadIdx.x; e < GM * GK; e += 256) {
            const int r = e / GK, c = e % GK;
            const int gk = k0 + c;
            As[c][r] = J[(long)(i0 + r) * ld + gk];
            const int gb = b0 + r;
            Bs[c][r] = (gb < B && gk < Nv) ? Q[(long)gb * Nv + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            double a[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ty * 4 + u];
                bv[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], bv[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gi = i0 + ty * 4 + u, gb = b0 + tx * 4 + w;
            if (gi < Nv && gb < B) Phi[(long)gb * Nv + gi] = acc[u][w];
        }
}

// One block per configuration: energy (with the counts penalty) and dE/dL.
// Phi row b starts at Phi + b * phi_ld (FP64 from the CUDA-core GEMM, FP32
// from the tensor-core path).
template <typename PT>
__global__ void k_grad_finish(const double* __restrict__ p, const double* __restrict__ q,
                              const PT* __restrict__ Phi, long phi_ld, const double* __restrict__ phifix,
                              const double* __restrict__ colsum, const int32_t* __restrict__ vclass,
                              const int32_t* __restrict__ counts, const double* __restrict__ z, int Nv, int S,
                              int ncls, double lambda, double E_const, double* __restrict__ E,
                              float* __restrict__ dlogits)
{
    __shared__ double red[256];
    const int b = blockIdx.x;
    const double* cb = colsum + (long)b * ncls * S;
    double acc = 0.0;
    for (int v = threadIdx.x; v < Nv; v += blockDim.x) {
        const long t = (long)b * Nv + v;
        const double jq = (double)Phi[(long)b * phi_ld + v] + phifix[v];     // (J q)_v over all sites
        acc += q[t] * (jq + phifix[v]);
        if (dlogits) {
            const int k = vclass[v];
            double g[64];
            double pg = 0.0;
            for (int s = 0; s < S; ++s) {
                g[s] = z[s] * 2.0 * jq + 2.0 * lambda * (cb[k * S + s] - counts[k * S + s]);
                pg += p[t * S + s] * g[s];
            }
            for (int s = 0; s < S; ++s)
                dlogits[t * S + s] = counts[k * S + s] > 0 ? (float)(p[t * S + s] * (g[s] - pg)) : 0.0f;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double pen = 0.0;
        for (int k = 0; k < ncls; ++k)
            for (int s = 0; s < S; ++s)
                if (counts[k * S + s] > 0) {
                    const double r = cb[k * S + s] - counts[k * S + s];
                    pen += r * r;
                }
        E[b] = red[0] + E_const + lambda * pen;
    }
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// q's hi / lo parts at element e of the two planes [2][plane]: TF32 in FP32
// storage, or FP16 of q qscale (F16), lo the rounding of what hi leaves.
template <bool F16>
__device__ __forceinline__ void store_q_planes(void* qt2, long plane, long e, float q, float qscale)
{
    if constexpr (F16) {
        q *= qscale;                           // a power of two: |q qscale| < 2^14
        __half* h = (__half*)qt2;
        const __half hi = __float2half_rn(q);
        h[e] = hi;
        h[plane + e] = __float2half_rn(q - __half2float(hi));
    } else {
        float* f = (float*)qt2;
        const float hi = tf32_rna(q);
        f[e] = hi;
        f[plane + e] = tf32_rna(q - hi);
    }
}

// p = softmax of the logits over the species allowed in the site's class, FP32 out.
__global__ void k_softmax_f32(const float* __restrict__ logits, long BN, int Nv, int S,
                              const int32_t* __restrict__ vclass, const int32_t* __restrict__ counts,
                              float* __restrict__ p)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= BN) return;
    const int k = vclass[(int)(t % Nv)];
    const float* L = logits + t * S;
    double m = -INFINITY;
    for (int s = 0; s < S; ++s)
        if (counts[k * S + s] > 0 && (double)L[s] > m) m = (double)L[s];
    double den = 0.0;
    for (int s = 0; s < S; ++s) den += counts[k * S + s] > 0 ? exp((double)L[s] - m) : 0.0;
    for (int s = 0; s < S; ++s) p[t * S + s] = counts[k * S + s] > 0 ? (float)(exp((double)L[s] - m) / den) : 0.0f;
}

// ---- tensor-core (TF32x2) path: FP32 elementwise chain ----------------------
// One pass over the padded operand: p = softmax of the logits over the
// species allowed in the site's class (FP32, B x Nv x S), q = sum_s p_s z_s,
// and q's TF32 hi / lo planes [2][Bpad][ld] for the contraction (zero padded).
template <bool F16>
__global__ void k_relax_prep(const float* __restrict__ logits, int B, int Nv, int S, int Bpad, int ld,
                             const int32_t* __restrict__ vclass, const int32_t* __restrict__ counts,
                             const double* __restrict__ z, float* __restrict__ p, void* __restrict__ qt2,
                             float qscale)
{
    const long plane = (long)Bpad * ld;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += (long)gridDim.x * blockDim.x) {
        const int b = (int)(e / ld), v = (int)(e % ld);
        float q = 0.0f;
        if (b < B && v < Nv) {
            const int k = vclass[v];
            const long t = (long)b * Nv + v;
            const float* L = logits + t * S;
            float m = -INFINITY;
            for (int s = 0; s < S; ++s)
                if (counts[k * S + s] > 0) m = fmaxf(m, L[s]);
            float den = 0.0f;
            for (int s = 0; s < S; ++s) den += counts[k * S + s] > 0 ? expf(L[s] - m) : 0.0f;
            const float inv = 1.0f / den;
            for (int s = 0; s < S; ++s) {
                const float ps = counts[k * S + s] > 0 ? expf(L[s] - m) * inv : 0.0f;
                p[t * S + s] = ps;
                q = fmaf(ps, (float)z[s], q);
            }
        }
        store_q_planes<F16>(qt2, plane, e, q, qscale);
    }
}

// colsum[(b*ncls + k)*S + s] = sum_{v in class k} p[b][v][s] from FP32 p, one
// block per (b, k) and one pass over the class's sites: each thread keeps FP32
// partial sums of all species (S <= 8) of its strided positions, then the block
// adds them in FP64 in a fixed order.  More species: one pass per species.
__global__ void __launch_bounds__(256) k_colsum_f32(const float* __restrict__ p, int Nv, int S, int ncls,
                                                    const int32_t* __restrict__ cls_start,
                                                    const int32_t* __restrict__ cls_pos, double* __restrict__ colsum)
{
    __shared__ double red[8][256];
    const int b = blockIdx.x / ncls, k = blockIdx.x % ncls;
    const int cs = cls_start[k], ce = cls_start[k + 1];
    if (S <= 8) {
        float a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = cs + threadIdx.x; i < ce; i += blockDim.x) {
            const float* pv = p + ((long)b * Nv + cls_pos[i]) * S;
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (s < S) a[s] += pv[s];
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) red[s][threadIdx.x] = (double)a[s];
        __syncthreads();
        for (int w = 128; w; w >>= 1) {
            if (threadIdx.x < w)
#pragma unroll
                for (int s = 0; s < 8; ++s) red[s][threadIdx.x] += red[s][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x < S) colsum[((long)b * ncls + k) * S + threadIdx.x] = red[threadIdx.x][0];
        return;
    }
    for (int s = 0; s < S; ++s) {
        float acc = 0.0f;
        for (int i = cs + threadIdx.x; i < ce; i += blockDim.x) acc += p[((long)b * Nv + cls_pos[i]) * S + s];
        red[0][threadIdx.x] = (double)acc;
        __syncthreads();
        for (int w = 128; w; w >>= 1) {
            if (threadIdx.x < w) red[0][threadIdx.x] += red[0][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) colsum[((long)b * ncls + k) * S + s] = red[0][0];
        __syncthreads();
    }
}

// One block per configuration, FP32 chain rule (q recomputed from p), energy
// accumulated in FP64: E_b = sum_v q_v (Phi_v + 2 phi_fix_v) + E_const + penalty.
// The per-(class, species) penalty terms 2 lambda (colsum - n) and the allowed
// mask are formed once per block (FP64, then FP32) in shared memory.
__global__ void __launch_bounds__(256) k_grad_finish_f32(const float* __restrict__ p, const float* __restrict__ Phi,
                                                         long phi_ld, const double* __restrict__ phifix,
                                                         const double* __restrict__ colsum,
                                                         const int32_t* __restrict__ vclass,
                                                         const int32_t* __restrict__ counts,
                                                         const double* __restrict__ z, int Nv, int S, int ncls,
                                                         double lambda, double E_const, double* __restrict__ E,
                                                         float* __restrict__ dlogits, float* logits_upd, float eta)
{
    constexpr int PEN_MAX = 512;                  // ncls * S entries held in shared memory
    __shared__ double red[256];
    __shared__ float zs[64];
    __shared__ float pen[PEN_MAX];
    __shared__ unsigned char allowed[PEN_MAX];
    const int b = blockIdx.x;
    const double* cb = colsum + (long)b * ncls * S;
    const int npen = ncls * S;
    if (threadIdx.x < 64) zs[threadIdx.x] = threadIdx.x < S ? (float)z[threadIdx.x] : 0.0f;
    for (int e = threadIdx.x; e < npen && e < PEN_MAX; e += blockDim.x) {
        pen[e] = (float)(2.0 * lambda * (cb[e] - counts[e]));
        allowed[e] = counts[e] > 0;
    }
    __syncthreads();
    const bool in_smem = npen <= PEN_MAX;
    double acc = 0.0;
    for (int v = threadIdx.x; v < Nv; v += blockDim.x) {
        const long t = (long)b * Nv + v;
        const float* pv = p + t * S;
        const float pf = (float)phifix[v];
        const float phi = Phi[(long)b * phi_ld + v];
        const float jq = phi + pf;                 // (J q)_v over all sites
        float q = 0.0f;
        for (int s = 0; s < S; ++s) q = fmaf(pv[s], zs[s], q);
        acc += (double)(q * (phi + 2.0f * pf));
        if (dlogits || logits_upd) {
            const int k = vclass[v];
            float pg = 0.0f;
            for (int s = 0; s < S; ++s) {
                const int e = k * S + s;
                const float pe = in_smem ? pen[e] : (float)(2.0 * lambda * (cb[e] - counts[e]));
                pg = fmaf(pv[s], fmaf(2.0f * zs[s], jq, pe), pg);
            }
            for (int s = 0; s < S; ++s) {
                const int e = k * S + s;
                const bool al = in_smem ? allowed[e] != 0 : counts[e] > 0;
                const float pe = in_smem ? pen[e] : (float)(2.0 * lambda * (cb[e] - counts[e]));
                const float g = al ? pv[s] * (fmaf(2.0f * zs[s], jq, pe) - pg) : 0.0f;
                if (dlogits) dlogits[t * S + s] = g;
                // descent step in place (this step's p was formed from the old logits)
                if (logits_upd) logits_upd[t * S + s] = logits_upd[t * S + s] - eta * g;
            }
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double pn = 0.0;
        for (int k = 0; k < ncls; ++k)
            for (int s = 0; s < S; ++s)
                if (counts[k * S + s] > 0) {
                    const double r = cb[k * S + s] - counts[k * S + s];
                    pn += r * r;
                }
        E[b] = red[0] + E_const + lambda * pn;
    }
}

// ---- vectorised fast path (S <= 8, ncls S <= 64, Nv % 4 == 0) ------------------
// The logits and p are B x Nv x S floats, so a thread that owns one site reads
// S floats 4 S bytes from its neighbour's and fetches every sector S times.
// Here a thread owns four consecutive sites of one configuration: their 4 S
// floats are S aligned float4 (the flattened site index b Nv + v is a multiple
// of 4), S is a template parameter so that all of them stay in registers, and
// Phi, phi_fix and the site classes of the four sites are one vector load each.
constexpr int RV_T = 256;                     // threads per block
constexpr int RV_G = 4;                       // sites per thread
constexpr int RV_C = RV_T * RV_G;             // sites per block (a chunk of one configuration's row)
constexpr int RV_SMAX = 8;
constexpr int RV_KS = 64;                     // ncls * S limit of the chunk partials

// One block per (configuration b < B, chunk c of 1,024 sites): p = softmax over
// the species allowed in the site's class, q = sum_s p_s z_s and q's TF32 hi /
// lo planes (zero for Nv <= v < ld; rows B .. Bpad are zeroed by the host), and
// the chunk's occupation sums cpart[(b nch + c) ncls S + k S + s] = sum over
// the chunk's sites v of class k of p_vs (FP32 within a thread and a warp in a
// fixed order, FP64 over the eight warps in order).
template <int S, bool F16>
__global__ void __launch_bounds__(RV_T) k_relax_prep_v4(const float* __restrict__ logits, int Nv, int ld, int nch,
                                                      const int32_t* __restrict__ vclass,
                                                      const int32_t* __restrict__ counts,
                                                      const double* __restrict__ z, int ncls, float* __restrict__ p,
                                                      void* __restrict__ qt2, long plane, double* __restrict__ cpart,
                                                      float qscale)
{
    __shared__ int cnt[RV_KS];
    __shared__ float zs[S];
    __shared__ double wsum[RV_T / 32][RV_KS];
    const int nks = ncls * S;
    if (threadIdx.x < nks) cnt[threadIdx.x] = counts[threadIdx.x];
    if (threadIdx.x < S) zs[threadIdx.x] = (float)z[threadIdx.x];   // once per block: conversions use the FP64 pipe
    __syncthreads();
    float zf[S];
#pragma unroll
    for (int t = 0; t < S; ++t) zf[t] = zs[t];
    const int c = blockIdx.x % nch, b = blockIdx.x / nch;
    const int v0 = c * RV_C + threadIdx.x * RV_G;
    const int nv = max(0, min(RV_G, Nv - v0));
    const long t0 = (long)b * Nv + v0;
    float P[RV_G * S];
    if (nv == RV_G) {
        const float4* src = reinterpret_cast<const float4*>(logits + t0 * S);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float4 f = src[j];
            P[4 * j] = f.x;
            P[4 * j + 1] = f.y;
            P[4 * j + 2] = f.z;
            P[4 * j + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < RV_G * S; ++j) P[j] = j < nv * S ? logits[t0 * S + j] : 0.0f;
    }
    int kc[RV_G];
    float qv[RV_G];
    if (nv == RV_G) {
        const int4 k4 = *reinterpret_cast<const int4*>(vclass + v0);
        kc[0] = k4.x;
        kc[1] = k4.y;
        kc[2] = k4.z;
        kc[3] = k4.w;
    } else {
#pragma unroll
        for (int g = 0; g < RV_G; ++g) kc[g] = g < nv ? vclass[v0 + g] : -1;
    }
#pragma unroll
    for (int g = 0; g < RV_G; ++g) {
        qv[g] = 0.0f;
        if (kc[g] >= 0) {
            const int k = kc[g];
            float m = -INFINITY;
#pragma unroll
            for (int t = 0; t < S; ++t)
                if (cnt[k * S + t] > 0) m = fmaxf(m, P[g * S + t]);
            float den = 0.0f;
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const float e = cnt[k * S + t] > 0 ? expf(P[g * S + t] - m) : 0.0f;
                P[g * S + t] = e;
                den += e;
            }
            const float inv = 1.0f / den;
#pragma unroll
            for (int t = 0; t < S; ++t) {
                P[g * S + t] *= inv;
                qv[g] = fmaf(P[g * S + t], zf[t], qv[g]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < S; ++t) P[g * S + t] = 0.0f;
        }
    }
    if (nv == RV_G) {
        float4* dst = reinterpret_cast<float4*>(p + t0 * S);
#pragma unroll
        for (int j = 0; j < S; ++j) dst[j] = make_float4(P[4 * j], P[4 * j + 1], P[4 * j + 2], P[4 * j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < RV_G * S; ++j)
            if (j < nv * S) p[t0 * S + j] = P[j];
    }
    if (v0 + RV_G <= ld) {
        if constexpr (F16) {
            __half2 hi[2], lo[2];
#pragma unroll
            for (int g = 0; g < RV_G; g += 2) {
                const float a0 = qv[g] * qscale, a1 = qv[g + 1] * qscale;   // a power of two: |a| < 2^14
                const __half h0 = __float2half_rn(a0), h1 = __float2half_rn(a1);
                hi[g / 2] = __halves2half2(h0, h1);
                lo[g / 2] = __halves2half2(__float2half_rn(a0 - __half2float(h0)), __float2half_rn(a1 - __half2float(h1)));
            }
            __half* h = (__half*)qt2;
            *reinterpret_cast<uint2*>(h + (long)b * ld + v0) = *reinterpret_cast<const uint2*>(hi);
            *reinterpret_cast<uint2*>(h + plane + (long)b * ld + v0) = *reinterpret_cast<const uint2*>(lo);
        } else {
            float hi[RV_G], lo[RV_G];
#pragma unroll
            for (int g = 0; g < RV_G; ++g) {
                hi[g] = tf32_rna(qv[g]);
                lo[g] = tf32_rna(qv[g] - hi[g]);
            }
            float* f = (float*)qt2;
            *reinterpret_cast<float4*>(f + (long)b * ld + v0) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(f + plane + (long)b * ld + v0) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int kk = 0; kk < ncls; ++kk)
#pragma unroll
        for (int t = 0; t < S; ++t) {
            float x = 0.0f;
#pragma unroll
            for (int g = 0; g < RV_G; ++g) x += kc[g] == kk ? P[g * S + t] : 0.0f;
#pragma unroll
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) wsum[warp][kk * S + t] = (double)x;
        }
    __syncthreads();
    if (threadIdx.x < nks) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < RV_T / 32; ++w) acc += wsum[w][threadIdx.x];
        cpart[((long)b * nch + c) * nks + threadIdx.x] = acc;
    }
}

// The FP32 chain rule of k_grad_finish_f32 for four sites per thread, one block
// per (configuration b, chunk c); colsum of b is the sum of its chunk partials
// in chunk order, and the block's share of the energy sum_v q_v (Phi_v +
// 2 phi_fix_v) goes to epart[b nch + c] (FP64, fixed order).
template <int S>
__global__ void __launch_bounds__(RV_T) k_grad_finish_v4(const float* __restrict__ p, const float* __restrict__ Phi,
                                                       long phi_ld, const float* __restrict__ phifixf,
                                                       const double* __restrict__ cpart, int nch,
                                                       const int32_t* __restrict__ vclass,
                                                       const int32_t* __restrict__ counts,
                                                       const double* __restrict__ z, int Nv, int ncls, double lambda,
                                                       double* __restrict__ epart, float* __restrict__ dlogits,
                                                       float* logits_upd, float eta)
{
    __shared__ float pen[RV_KS];
    __shared__ int cnt[RV_KS];
    __shared__ float zs[S];
    __shared__ double red[RV_T / 32];
    const int c = blockIdx.x % nch, b = blockIdx.x / nch;
    const int nks = ncls * S;
    if (threadIdx.x < nks) {
        double a = 0.0;
        for (int cc = 0; cc < nch; ++cc) a += cpart[((long)b * nch + cc) * nks + threadIdx.x];
        cnt[threadIdx.x] = counts[threadIdx.x];
        pen[threadIdx.x] = (float)(2.0 * lambda * (a - counts[threadIdx.x]));
    }
    if (threadIdx.x < S) zs[threadIdx.x] = (float)z[threadIdx.x];   // once per block: conversions use the FP64 pipe
    __syncthreads();
    float zf[S];
#pragma unroll
    for (int t = 0; t < S; ++t) zf[t] = zs[t];
    const int v0 = c * RV_C + threadIdx.x * RV_G;
    const int nv = max(0, min(RV_G, Nv - v0));
    const long t0 = (long)b * Nv + v0;
    float P[RV_G * S];
    float phi[RV_G], pf[RV_G];
    int kc[RV_G];
    if (nv == RV_G) {
        const float4* src = reinterpret_cast<const float4*>(p + t0 * S);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float4 f = src[j];
            P[4 * j] = f.x;
            P[4 * j + 1] = f.y;
            P[4 * j + 2] = f.z;
            P[4 * j + 3] = f.w;
        }
        const float4 f = *reinterpret_cast<const float4*>(Phi + (long)b * phi_ld + v0);
        phi[0] = f.x;
        phi[1] = f.y;
        phi[2] = f.z;
        phi[3] = f.w;
        const float4 f4 = *reinterpret_cast<const float4*>(phifixf + v0);
        pf[0] = f4.x;
        pf[1] = f4.y;
        pf[2] = f4.z;
        pf[3] = f4.w;
        const int4 k4 = *reinterpret_cast<const int4*>(vclass + v0);
        kc[0] = k4.x;
        kc[1] = k4.y;
        kc[2] = k4.z;
        kc[3] = k4.w;
    } else {
#pragma unroll
        for (int j = 0; j < RV_G * S; ++j) P[j] = j < nv * S ? p[t0 * S + j] : 0.0f;
#pragma unroll
        for (int g = 0; g < RV_G; ++g) {
            phi[g] = g < nv ? Phi[(long)b * phi_ld + v0 + g] : 0.0f;
            pf[g] = g < nv ? phifixf[v0 + g] : 0.0f;
            kc[g] = g < nv ? vclass[v0 + g] : -1;
        }
    }
    // the four sites' energy terms summed in FP32, the threads' sums in FP64 (conversions and FP64
    // additions run on GB300's narrow FP64 pipe: one per thread, not one per site)
    float accf = 0.0f;
    const bool grad = dlogits || logits_upd;
    float G[RV_G * S];
#pragma unroll
    for (int g = 0; g < RV_G; ++g) {
        float q = 0.0f;
#pragma unroll
        for (int t = 0; t < S; ++t) q = fmaf(P[g * S + t], zf[t], q);
        accf += q * (phi[g] + 2.0f * pf[g]);
        const int k = kc[g] < 0 ? 0 : kc[g];
        const float jq = phi[g] + pf[g];           // (J q)_v over all sites
        float pg = 0.0f;
#pragma unroll
        for (int t = 0; t < S; ++t) pg = fmaf(P[g * S + t], fmaf(2.0f * zf[t], jq, pen[k * S + t]), pg);
#pragma unroll
        for (int t = 0; t < S; ++t)
            G[g * S + t] = cnt[k * S + t] > 0 ? P[g * S + t] * (fmaf(2.0f * zf[t], jq, pen[k * S + t]) - pg) : 0.0f;
    }
    if (grad && nv == RV_G) {
        if (dlogits) {
            float4* dst = reinterpret_cast<float4*>(dlogits + t0 * S);
#pragma unroll
            for (int j = 0; j < S; ++j) dst[j] = make_float4(G[4 * j], G[4 * j + 1], G[4 * j + 2], G[4 * j + 3]);
        }
        if (logits_upd) {
            // descent step in place (this step's p was formed from the old logits)
            float4* dst = reinterpret_cast<float4*>(logits_upd + t0 * S);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                float4 f = dst[j];
                f.x -= eta * G[4 * j];
                f.y -= eta * G[4 * j + 1];
                f.z -= eta * G[4 * j + 2];
                f.w -= eta * G[4 * j + 3];
                dst[j] = f;
            }
        }
    } else if (grad) {
#pragma unroll
        for (int j = 0; j < RV_G * S; ++j)
            if (j < nv * S) {
                if (dlogits) dlogits[t0 * S + j] = G[j];
                if (logits_upd) logits_upd[t0 * S + j] = logits_upd[t0 * S + j] - eta * G[j];
            }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = (double)accf;
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
#pragma unroll
        for (int w = 0; w < RV_T / 32; ++w) e += red[w];
        epart[(long)b * nch + blockIdx.x % nch] = e;
    }
}

// E_b = sum_c epart[b nch + c] + E_const + lambda sum_{k,s allowed} (colsum - n)^2,
// colsum summed from the chunk partials in chunk order; one thread per configuration.
__global__ void k_energy_v4(const double* __restrict__ epart, const double* __restrict__ cpart, int nch, int B,
                            int ncls, int S, const int32_t* __restrict__ counts, double lambda, double E_const,
                            double* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int nks = ncls * S;
    double e = 0.0;
    for (int c = 0; c < nch; ++c) e += epart[(long)b * nch + c];
    double pn = 0.0;
    for (int i = 0; i < nks; ++i) {
        if (counts[i] <= 0) continue;
        double a = 0.0;
        for (int c = 0; c < nch; ++c) a += cpart[((long)b * nch + c) * nks + i];
        const double r = a - counts[i];
        pn += r * r;
    }
    E[b] = e + E_const + lambda * pn;
}

template <int S>
void launch_relax_v4(int B, int Nv, int ld, int nch, const goac_problem* p, const float* logits, float* P32,
                     void* qt2, long plane, double* cpart, bool f16, float qscale, cudaStream_t st)
{
    if (f16)
        goac::launch(k_relax_prep_v4<S, true>, B * nch, RV_T, 0, st, logits, Nv, ld, nch, (const int32_t*)p->vclass_dev,
                     (const int32_t*)p->counts_dev, (const double*)p->z_dev, p->ncls, P32, qt2, plane, cpart, qscale);
    else
        goac::launch(k_relax_prep_v4<S, false>, B * nch, RV_T, 0, st, logits, Nv, ld, nch,
                     (const int32_t*)p->vclass_dev, (const int32_t*)p->counts_dev, (const double*)p->z_dev, p->ncls,
                     P32, qt2, plane, cpart, 1.0f);
}

template <int S>
void launch_finish_v4(int B, int Nv, int nch, int ld, const goac_problem* p, const float* P32, const float* Phi,
                      const double* cpart, double* epart, double lambda, float* dlogits, float* logits_upd, float eta,
                      cudaStream_t st)
{
    goac::launch(k_grad_finish_v4<S>, B * nch, RV_T, 0, st, P32, Phi, (long)ld, (const float*)p->phifix_f32, cpart, nch,
                 (const int32_t*)p->vclass_dev, (const int32_t*)p->counts_dev, (const double*)p->z_dev, Nv, p->ncls,
                 lambda, epart, dlogits, logits_upd, eta);
}

// out = (float) in.
__global__ void k_to_f32(const double* __restrict__ in, long n, float* __restrict__ out)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        out[e] = (float)in[e];
}

// L -= eta * dL (FP32, in place).
__global__ void k_descent_step(float* __restrict__ L, const float* __restrict__ dL, long n, float eta)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        L[e] = L[e] - eta * dL[e];
}

// ---- rounding to counts ------------------------------------------------------
// Sort key of a (site v, species s) pair: p descending, then v, then s ascending.
__device__ __forceinline__ unsigned long long pair_key(float pv, int v, int s)
{
    return ((unsigned long long)(~__float_as_uint(pv)) << 32) | ((unsigned long long)(uint32_t)v << 8) | (uint32_t)s;
}

__global__ void k_round_keys(const float* __restrict__ p, int Nv, int S, int ncls, const int32_t* __restrict__ cls_start,
                             const int32_t* __restrict__ cls_pos, const int32_t* __restrict__ counts,
                             const long long* __restrict__ seg_off, const int* __restrict__ seg_M, long long per_b,
                             unsigned long long* __restrict__ keys)
{
    const int b = blockIdx.x / ncls, k = blockIdx.x % ncls;
    const int cs = cls_start[k], n = cls_start[k + 1] - cs;
    int allowed[64];
    int na = 0;
    for (int s = 0; s < S; ++s)
        if (counts[k * S + s] > 0) allowed[na++] = s;
    unsigned long long* out = keys + (long long)b * per_b + seg_off[k];
    const int M = seg_M[k];
    const long m = (long)n * na;
    for (long e = threadIdx.x; e < M; e += blockDim.x) {
        if (e < m) {
            const int v = cls_pos[cs + (int)(e / na)];
            const int s = allowed[e % na];
            out[e] = pair_key(p[((long)b * Nv + v) * S + s], v, s);
        } else {
            out[e] = ~0ull;
        }
    }
}

// Bitonic sort of each (configuration, class) segment, one block per segment.
__global__ void __launch_bounds__(1024) k_bitonic(unsigned long long* __restrict__ keys, int ncls,
                                                  const long long* __restrict__ seg_off, const int* __restrict__ seg_M,
                                                  long long per_b)
{
    const int b = blockIdx.x / ncls, k = blockIdx.x % ncls;
    unsigned long long* a = keys + (long long)b * per_b + seg_off[k];
    const int M = seg_M[k];
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < M; i += blockDim.x) {
                const int l = i ^ stride;
                if (l > i) {
                    const unsigned long long x = a[i], y = a[l];
                    const bool up = (i & size) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void k_round_greedy(const unsigned long long* __restrict__ keys, int B, int Nv, int S, int ncls,
                               const int32_t* __restrict__ cls_start, const int32_t* __restrict__ counts,
                               const long long* __restrict__ seg_off, long long per_b, int8_t* __restrict__ species,
                               int* __restrict__ err)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * ncls) return;
    const int b = (int)(t / ncls), k = (int)(t % ncls);
    const int n = cls_start[k + 1] - cls_start[k];
    int na = 0;
    int left[64];
    for (int s = 0; s < S; ++s) {
        left[s] = counts[k * S + s];
        na += left[s] > 0;
    }
    const unsigned long long* a = keys + (long long)b * per_b + seg_off[k];
    const long m = (long)n * na;
    int8_t* sp = species + (long)b * Nv;
    int placed = 0;
    for (long r = 0; r < m && placed < n; ++r) {
        const unsigned long long key = a[r];
        const int v = (int)((key & 0xffffffffull) >> 8);
        const int s = (int)(key & 0xffull);
        if (sp[v] >= 0 || left[s] == 0) continue;
        sp[v] = (int8_t)s;
        left[s]--;
        placed++;
    }
    if (placed != n) goacd::report(err, GOAC_ERR_INTERNAL, goac::SITE_ROUND, (int)t);
}

}  // namespace

// Energies and dE/dL (dlogits_dev, nullable); with logits_upd (TF32x2 only) the
// chain-rule kernel also applies L -= eta dE/dL in place, so that a descent step
// needs no separate pass over the gradient.
static goac_status energy_grad_impl(goac_problem* p, const float* logits_dev, int32_t B, double lambda,
                                    int32_t precision, double* E_dev, float* dlogits_dev, float* logits_upd,
                                    float eta);

extern "C" goac_status goac_energy_grad(goac_problem* p, const float* logits_dev, int32_t B, double lambda,
                                        int32_t precision, double* E_dev, float* dlogits_dev)
{
    return energy_grad_impl(p, logits_dev, B, lambda, precision, E_dev, dlogits_dev, nullptr, 0.0f);
}

static goac_status energy_grad_impl(goac_problem* p, const float* logits_dev, int32_t B, double lambda,
                                    int32_t precision, double* E_dev, float* dlogits_dev, float* logits_upd,
                                    float eta)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_energy_grad: NULL problem");
    if (B <= 0 || B > GOAC_MAX_BATCH)
        return B == 0 ? GOAC_OK : goac::fail(GOAC_ERR_INVALID_ARG, "goac_energy_grad: B < 0 or B > GOAC_MAX_BATCH");
    if (!logits_dev || !E_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_energy_grad: NULL");
    if (precision != GOAC_PREC_F64 && precision != GOAC_PREC_TF32X2 && precision != GOAC_PREC_F16X2)
        return goac::fail(GOAC_ERR_UNSUPPORTED, "goac_energy_grad: precision must be F64, TF32X2 or F16X2");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const int Nv = p->Nv, S = p->S, ncls = p->ncls, ld = p->Nv_pad;
    const bool tc = precision == GOAC_PREC_TF32X2 || precision == GOAC_PREC_F16X2;
    const bool f16 = precision == GOAC_PREC_F16X2;
    const size_t qbytes = f16 ? sizeof(__half) : sizeof(float);   // one element of q's hi / lo planes
    // FP16: q is scaled by 2^qshift so that |q| 2^qshift < 2^14 (|q| <= max |z|), and so that the lo
    // parts of all but the smallest charges stay in FP16's normal range; the contraction undoes it
    int qshift = 0;
    if (f16) {
        double zmax = 0.0;
        for (int s2 = 0; s2 < S; ++s2) zmax = std::max(zmax, fabs(p->z[s2]));
        int ez = 0;
        if (zmax > 0.0) frexp(zmax, &ez);         // zmax < 2^ez
        qshift = 14 - ez;
    }
    const float qscale = (float)ldexp(1.0, qshift);
    const int Bpad = ((B + 255) / 256) * 256;      // whole 256-configuration tiles of the contraction
    const long BN = (long)B * Nv;
    cudaStream_t st = p->ctx->stream;
    if (tc) {
        // FP32 elementwise chain around the TF32x2 contraction
        // four sites per thread for up to 8 species, 64 (class, species) pairs and Nv % 4 == 0 with
        // 16-byte aligned logits / gradient arrays; else one site per thread
        const bool a16 = ((uintptr_t)logits_dev & 15) == 0 && ((uintptr_t)dlogits_dev & 15) == 0 &&
                         ((uintptr_t)logits_upd & 15) == 0;
        const bool vec = S <= RV_SMAX && ncls * S <= RV_KS && Nv % 4 == 0 && a16;
        const int nch = (Nv + RV_C - 1) / RV_C;
        const size_t ncol = vec ? (size_t)B * nch * ncls * S + (size_t)B * nch : (size_t)B * ncls * S;
        size_t need = sizeof(float) * (size_t)BN * S + sizeof(double) * ncol + sizeof(float) * 3 * (size_t)Bpad * ld +
                      1024;
        goac_status rc = goac::ensure(p->grad_tmp, need);
        if (rc) return rc;
        float* P32 = (float*)p->grad_tmp.ptr;
        double* colsum = (double*)(((uintptr_t)(P32 + BN * S) + 255) & ~(uintptr_t)255);
        double* epart = colsum + (size_t)B * nch * ncls * S;        // vec only
        float* qt2f = (float*)(((uintptr_t)(colsum + ncol) + 255) & ~(uintptr_t)255);   // TMA: aligned
        void* qt2 = qt2f;                                       // FP32 planes, or FP16 planes in their front half
        float* Phi = qt2f + 2 * (size_t)Bpad * ld;
        const long plane = (long)Bpad * ld;
        if (vec && !p->phifix_f32) {
            GOAC_CUDA(cudaMalloc(&p->phifix_f32, sizeof(float) * (size_t)ld));
            goac::launch(k_to_f32, (ld + 255) / 256, 256, 0, st, (const double*)p->phifix, (long)ld, p->phifix_f32);
        }
        if (vec) {
            if (Bpad > B) {
                uint8_t* q8 = (uint8_t*)qt2;
                GOAC_CUDA(cudaMemsetAsync(q8 + qbytes * (size_t)B * ld, 0, qbytes * (size_t)(Bpad - B) * ld, st));
                GOAC_CUDA(cudaMemsetAsync(q8 + qbytes * ((size_t)plane + (size_t)B * ld), 0,
                                          qbytes * (size_t)(Bpad - B) * ld, st));
            }
            switch (S) {
            case 1: launch_relax_v4<1>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 2: launch_relax_v4<2>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 3: launch_relax_v4<3>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 4: launch_relax_v4<4>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 5: launch_relax_v4<5>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 6: launch_relax_v4<6>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            case 7: launch_relax_v4<7>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            default: launch_relax_v4<8>(B, Nv, ld, nch, p, logits_dev, P32, qt2, plane, colsum, f16, qscale, st); break;
            }
        } else {
            if (f16)
                goac::launch(k_relax_prep<true>, (int)std::min<long>((plane + 255) / 256, 65535L * 4), 256, 0, st,
                             logits_dev, B, Nv, S, Bpad, ld, p->vclass_dev, p->counts_dev, p->z_dev, P32, qt2,
                             qscale);
            else
                goac::launch(k_relax_prep<false>, (int)std::min<long>((plane + 255) / 256, 65535L * 4), 256, 0, st,
                             logits_dev, B, Nv, S, Bpad, ld, p->vclass_dev, p->counts_dev, p->z_dev, P32, qt2, 1.0f);
            goac::launch(k_colsum_f32, B * ncls, 256, 0, st, (const float*)P32, Nv, S, ncls, p->cls_start_dev,
                         p->cls_pos_dev, colsum);
        }
        GOAC_LAUNCH_CHECK("k_relax_prep");
        rc = goac::phi_tc(p, qt2, Bpad, Phi, f16, qshift);
        if (rc) return rc;
        if (vec) {
#define GOAC_FINISH_V4(SS)                                                                                         \
    launch_finish_v4<SS>(B, Nv, nch, ld, p, P32, Phi, colsum, epart, lambda, dlogits_dev, logits_upd, eta, st)
            switch (S) {
            case 1: GOAC_FINISH_V4(1); break;
            case 2: GOAC_FINISH_V4(2); break;
            case 3: GOAC_FINISH_V4(3); break;
            case 4: GOAC_FINISH_V4(4); break;
            case 5: GOAC_FINISH_V4(5); break;
            case 6: GOAC_FINISH_V4(6); break;
            case 7: GOAC_FINISH_V4(7); break;
            default: GOAC_FINISH_V4(8); break;
            }
#undef GOAC_FINISH_V4
            goac::launch(k_energy_v4, (B + 255) / 256, 256, 0, st, (const double*)epart, (const double*)colsum, nch, B,
                         ncls, S, p->counts_dev, lambda, p->E_const, E_dev);
        } else {
            goac::launch(k_grad_finish_f32, B, 256, 0, st, (const float*)P32, (const float*)Phi, (long)ld,
                         (const double*)p->phifix, (const double*)colsum, p->vclass_dev, p->counts_dev, p->z_dev, Nv,
                         S, ncls, lambda, p->E_const, E_dev, dlogits_dev, logits_upd, eta);
        }
    } else {
        size_t need = sizeof(double) * ((size_t)BN * S + (size_t)BN + (size_t)B * ncls * S + (size_t)BN) + 2048;
        goac_status rc = goac::ensure(p->grad_tmp, need);
        if (rc) return rc;
        double* P_ = (double*)p->grad_tmp.ptr;
        double* Q = P_ + BN * S;
        double* colsum = Q + BN;
        double* Phi = colsum + (long)B * ncls * S;
        goac::launch(k_softmax, (int)((BN + 255) / 256), 256, 0, st, logits_dev, BN, Nv, S, p->vclass_dev,
                     p->counts_dev, p->z_dev, P_, Q);
        goac::launch(k_colsum, B * ncls, 256, 0, st, P_, Nv, S, ncls, p->cls_start_dev, p->cls_pos_dev, colsum);
        dim3 grid((B + GM - 1) / GM, (Nv + GM - 1) / GM);
        goac::launch(k_phi_real, grid, 256, 0, st, (const double*)p->J_vv, ld, Nv, (const double*)Q, B, Phi);
        goac::launch(k_grad_finish<double>, B, 256, 0, st, (const double*)P_, (const double*)Q, (const double*)Phi,
                     (long)Nv, (const double*)p->phifix, (const double*)colsum, p->vclass_dev, p->counts_dev,
                     p->z_dev, Nv, S, ncls, lambda, p->E_const, E_dev, dlogits_dev);
    }
    GOAC_LAUNCH_CHECK("goac_energy_grad");
    return GOAC_OK;
}

extern "C" goac_status goac_round_to_counts(goac_problem* p, const float* p_dev, int32_t B, int8_t* species_dev)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_round_to_counts: NULL problem");
    if (B <= 0 || B > GOAC_MAX_BATCH)
        return B == 0 ? GOAC_OK : goac::fail(GOAC_ERR_INVALID_ARG, "goac_round_to_counts: B < 0 or B > GOAC_MAX_BATCH");
    if (!p_dev || !species_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_round_to_counts: NULL");
    if (p->Nv >= (1 << 24)) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_round_to_counts: Nv too large");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const int ncls = p->ncls, S = p->S;
    std::vector<long long> off(ncls);
    std::vector<int> Ms(ncls);
    long long per_b = 0;
    for (int k = 0; k < ncls; ++k) {
        int na = 0;
        for (int s = 0; s < S; ++s) na += p->counts[k * S + s] > 0;
        const long m = (long)(p->cls_start[k + 1] - p->cls_start[k]) * na;
        int M = 1;
        while (M < m) M <<= 1;
        if (M > (1 << 26)) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_round_to_counts: class too large");
        off[k] = per_b;
        Ms[k] = M;
        per_b += M;
    }
    const size_t keys_bytes = sizeof(unsigned long long) * (size_t)per_b * B;
    goac_status rc = goac::ensure(p->grad_tmp, keys_bytes + sizeof(long long) * ncls + sizeof(int) * ncls + 64);
    if (rc) return rc;
    unsigned long long* keys = (unsigned long long*)p->grad_tmp.ptr;
    long long* d_off = (long long*)((char*)p->grad_tmp.ptr + keys_bytes);
    int* d_M = (int*)(d_off + ncls);
    cudaStream_t st = p->ctx->stream;
    GOAC_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * ncls, cudaMemcpyHostToDevice, st));
    GOAC_CUDA(cudaMemcpyAsync(d_M, Ms.data(), sizeof(int) * ncls, cudaMemcpyHostToDevice, st));
    GOAC_CUDA(cudaMemsetAsync(species_dev, 0xff, (size_t)B * p->Nv, st));
    goac::launch(k_round_keys, B * ncls, 256, 0, st, p_dev, p->Nv, S, ncls, p->cls_start_dev, p->cls_pos_dev, p->counts_dev, d_off,
                                           d_M, per_b, keys);
    goac::launch(k_bitonic, B * ncls, 1024, 0, st, keys, ncls, d_off, d_M, per_b);
    const long nt = (long)B * ncls;
    goac::launch(k_round_greedy, (int)((nt + 127) / 128), 128, 0, st, keys, B, p->Nv, S, ncls, p->cls_start_dev, p->counts_dev,
                                                            d_off, per_b, species_dev, p->ctx->d_err);
    GOAC_LAUNCH_CHECK("goac_round_to_counts");
    return GOAC_OK;
}

extern "C" goac_status goac_relaxed_descent(goac_problem* p, float* logits_dev, int32_t B, double lambda, double eta,
                                            int32_t n_steps, int32_t precision, float* dlogits_scratch_dev,
                                            double* E_dev)
{
    if (!p || B < 0 || B > GOAC_MAX_BATCH || n_steps < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_relaxed_descent: bad argument");
    if (B == 0) return GOAC_OK;
    if (!logits_dev || !dlogits_scratch_dev || !E_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_relaxed_descent: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const long n = (long)B * p->Nv * p->S;
    const int blocks = (int)std::min<long>((n + 255) / 256, 65535L * 4);
    for (int it = 0; it < n_steps; ++it) {
        if (precision == GOAC_PREC_TF32X2 || precision == GOAC_PREC_F16X2) {
            // gradient and step fused: the chain-rule kernel updates the logits in place
            goac_status rc = energy_grad_impl(p, logits_dev, B, lambda, precision, E_dev, nullptr, logits_dev, (float)eta);
            if (rc) return rc;
            continue;
        }
        goac_status rc = goac_energy_grad(p, logits_dev, B, lambda, precision, E_dev, dlogits_scratch_dev);
        if (rc) return rc;
        goac::launch(k_descent_step, blocks, 256, 0, p->ctx->stream, logits_dev, (const float*)dlogits_scratch_dev, n,
                     (float)eta);
        GOAC_LAUNCH_CHECK("k_descent_step");
    }
    return goac_energy_grad(p, logits_dev, B, lambda, precision, E_dev, nullptr);
}

extern "C" goac_status goac_occupations(goac_problem* p, const float* logits_dev, int32_t B, float* p_dev)
{
    if (!p || B < 0 || B > GOAC_MAX_BATCH) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_occupations: bad argument");
    if (B == 0) return GOAC_OK;
    if (!logits_dev || !p_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_occupations: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const long BN = (long)B * p->Nv;
    goac::launch(k_softmax_f32, (int)((BN + 255) / 256), 256, 0, p->ctx->stream, logits_dev, BN, p->Nv, p->S,
                 (const int32_t*)p->vclass_dev, (const int32_t*)p->counts_dev, p_dev);
    GOAC_LAUNCH_CHECK("k_softmax_f32");
    return GOAC_OK;
}
