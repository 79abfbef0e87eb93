// Gradient descent over single-swap neighbours (SI, Gradient Descent: all
// neighbouring solutions reachable by one swap are evaluated and the lowest
// energy one is taken until none is lower), for a batch of configurations.
//
// Per step and configuration: dE(a, b) = 2 d (phi_a - phi_b) + d^2 (J_aa + J_bb
// - 2 J_ab), d = q_b - q_a, over every pair a < b of the same class holding
// different species.  Pass 0 finds dmin; a configuration with dmin >= -1e-9 eV
// is at a local minimum.  Pass 1 finds the lowest pair (a, b) (lexicographic)
// with dE <= dmin + 1e-9 eV (ties within rounding resolve by index), which is
// then swapped: phi += d (J_:a - J_:b), E += dE.
//
// The pair scan is a tile computation over the upper triangle of 64 x 64
// blocks of J_vv: each CTA stages its J tile (doubled: 2 J_ab, exact) in
// shared memory once and evaluates it for GD_CFG configurations, with 2d and
// d^2 taken from a per-species-pair table.  Pass 0 filters in FP32 and decides
// in FP64: every pair's dE is formed in FP32 with a bound e on its distance
// from the FP64 value (a multiple of 2^-24 of the magnitudes that enter it);
// with U the least dE32 + e of the tile, only the pairs with dE32 - e <=
// U + 1e-9 eV can be the tile's minimum or lie within 1e-9 eV of it, and
// those few are evaluated again in FP64 with the definition's roundings, so
// the tile minimum and its tie set (its pairs within 1e-9 eV of the minimum,
// up to GK of them) are exactly those of an FP64 scan.  The pairs eligible in
// pass 1 all lie in the tie sets of the tiles whose minimum is within 1e-9 eV
// of dmin, so pass 1 (an FP64 scan of every pair) runs for a configuration
// only when one of those tie sets overflowed.  Per-tile candidates are reduced
// per configuration in a fixed order.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int GT = 64;        // tile edge (sites)
constexpr int GD_CFG = 4;     // configurations per CTA
constexpr int GK = 4;         // tie-set entries kept per tile and configuration
constexpr int GS = 16;        // species of the (2d, d^2) table (more: formed per pair)
constexpr double kTie = 1e-9; // energy tie tolerance (eV)

struct GdArgs {
    const double* J;          // Nv_pad x ld
    const double* diag;       // Nv
    const int8_t* species;    // B x Nv
    const double* phi;        // B x Nv
    const int32_t* vclass;    // Nv
    const double* z;          // 64
    const int* active;        // B
    const double* dmin;       // B (pass 1)
    const int* need1;         // B: pass 1 needed (a tie set overflowed)
    double* cand_val;         // ntiles x B: tile minimum (pass 0)
    unsigned long long* cand_key;   // ntiles x B (pass 1)
    double* tie_val;          // ntiles x B x GK: tie-set energies (pass 0)
    unsigned long long* tie_key;    // ntiles x B x GK: tie-set pair keys a Nv + b
    int* tie_n;               // ntiles x B: tie-set size (> GK: overflow)
    const float* J2f;         // Nv_pad x ld: 2 J_vv rounded to FP32 (pass 0's filter)
    const float* diagf;       // Nv: diag rounded to FP32
    float* phif;              // B x Nv: phi rounded to FP32, kept beside phi
    int ld, Nv, B, ntiles, S;
};

// FP32 copies for the filter of pass 0: 2 J (once per run) and the diagonal.
__global__ void k_gd_f32_consts(const double* __restrict__ J, long n, const double* __restrict__ diag, int Nv,
                                float* __restrict__ J2f, float* __restrict__ diagf)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        J2f[e] = (float)(2.0 * J[e]);
        if (e < Nv) diagf[e] = (float)diag[e];
    }
}

__global__ void k_gd_f32_phi(const double* __restrict__ phi, long n, float* __restrict__ phif)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        phif[e] = (float)phi[e];
}

__device__ __forceinline__ double pair_dE(double d, double pa, double pb, double jaa, double jbb, double jab)
{
    return __dadd_rn(__dmul_rn(__dmul_rn(2.0, d), __dsub_rn(pa, pb)),
                     __dmul_rn(__dmul_rn(d, d), __dsub_rn(__dadd_rn(jaa, jbb), __dmul_rn(2.0, jab))));
}

// dE with c1 = 2 d and c2 = d d (both as the definition rounds them) and
// jab2 = 2 J_ab: the same value as pair_dE, bit for bit.
__device__ __forceinline__ double pair_dE_c(double c1, double c2, double pa, double pb, double jaa, double jbb,
                                            double jab2)
{
    return __dadd_rn(__dmul_rn(c1, __dsub_rn(pa, pb)), __dmul_rn(c2, __dsub_rn(__dadd_rn(jaa, jbb), jab2)));
}

// Upper triangle tile t -> (row block bi, column block bj), bi <= bj.
__device__ __forceinline__ void gd_tile(int t, int& bi, int& bj)
{
    bj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
    while (bj * (bj + 1) / 2 > t) --bj;
    bi = t - bj * (bj + 1) / 2;
}

// Pass 0: FP32 filter, FP64 decision (see the top of the file).  Per pair the
// FP32 value is c1 (p_a - p_b) + c2 ((j_aa + j_bb) - 2 j_ab) from FP32 copies;
// each of its five roundings and each rounding of an input to FP32 moves it by
// at most 2^-24 of the magnitudes involved, and the bound e = 2^-19 (|c1|
// (|p_a| + |p_b|) + |c2| (|j_aa| + |j_bb| + |2 j_ab|)) + 2^-20 |dE32| also
// covers the FP32 roundings of the comparisons below (the threshold carries
// 2^-20 |U| for the same reason).
__global__ void __launch_bounds__(256, 4) k_gd_pass0(GdArgs g)
{
    __shared__ float Jf[GT][GT + 1];
    __shared__ double phI[GD_CFG][GT], phJ[GD_CFG][GT];
    __shared__ float pfI[GD_CFG][GT], pfJ[GD_CFG][GT];
    __shared__ int8_t spI[GD_CFG][GT], spJ[GD_CFG][GT];
    __shared__ int clI[GT], clJ[GT];
    __shared__ double dgI[GT], dgJ[GT];
    __shared__ float dfI[GT], dfJ[GT];
    __shared__ double c1t[GS * GS], c2t[GS * GS];
    __shared__ float c1f[GS * GS], c2f[GS * GS];
    __shared__ float redf[8];
    __shared__ double redv[8];
    __shared__ double tv[GK];
    __shared__ unsigned long long tk[GK];
    __shared__ int tn, tover;
    const int c0 = blockIdx.y * GD_CFG;
    int bi, bj;
    gd_tile(blockIdx.x, bi, bj);
    const int i0 = bi * GT, j0 = bj * GT;
    // FP32 copies staged as they are (FP64 to FP32 conversions run on GB300's FP64 pipe);
    // the FP64 values only for the candidates
    for (int e = threadIdx.x; e < GT * GT; e += 256) {
        const int r = e / GT, c = e % GT;
        Jf[r][c] = g.J2f[(long)(i0 + r) * g.ld + j0 + c];
    }
    const bool table = g.S <= GS;
    if (table)
        for (int e = threadIdx.x; e < g.S * g.S; e += 256) {
            const double d = __dsub_rn(g.z[e % g.S], g.z[e / g.S]);     // [sa][sb]: z_sb - z_sa
            c1t[e] = __dmul_rn(2.0, d);
            c2t[e] = __dmul_rn(d, d);
            c1f[e] = (float)c1t[e];
            c2f[e] = (float)c2t[e];
        }
    for (int e = threadIdx.x; e < GT; e += 256) {
        const bool vi = i0 + e < g.Nv, vj = j0 + e < g.Nv;
        clI[e] = vi ? g.vclass[i0 + e] : -1;
        clJ[e] = vj ? g.vclass[j0 + e] : -2;
        dgI[e] = vi ? g.diag[i0 + e] : 0.0;
        dgJ[e] = vj ? g.diag[j0 + e] : 0.0;
        dfI[e] = vi ? g.diagf[i0 + e] : 0.0f;
        dfJ[e] = vj ? g.diagf[j0 + e] : 0.0f;
    }
    for (int e = threadIdx.x; e < GD_CFG * GT; e += 256) {
        const int c = e / GT, x = e % GT, b = c0 + c;
        const bool okb = b < g.B;
        const bool vi = okb && i0 + x < g.Nv, vj = okb && j0 + x < g.Nv;
        phI[c][x] = vi ? g.phi[(long)b * g.Nv + i0 + x] : 0.0;
        phJ[c][x] = vj ? g.phi[(long)b * g.Nv + j0 + x] : 0.0;
        pfI[c][x] = vi ? g.phif[(long)b * g.Nv + i0 + x] : 0.0f;
        pfJ[c][x] = vj ? g.phif[(long)b * g.Nv + j0 + x] : 0.0f;
        spI[c][x] = vi ? g.species[(long)b * g.Nv + i0 + x] : (int8_t)-1;
        spJ[c][x] = vj ? g.species[(long)b * g.Nv + j0 + x] : (int8_t)-1;
    }
    __syncthreads();
    const int ii = threadIdx.x % GT;
    const int jq = (threadIdx.x / GT) * 16;
    const int a = i0 + ii;
    for (int c = 0; c < GD_CFG; ++c) {
        const int b = c0 + c;
        const bool live = b < g.B && g.active[b];   // uniform over the block
        if (!live) continue;
        const int sa = spI[c][ii];
        float lo[16];                              // dE32 - e (INFINITY: no pair)
        float ub = INFINITY;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int jj = jq + u;
            lo[u] = INFINITY;
            if (!(a < j0 + jj) || clI[ii] != clJ[jj]) continue;
            const int sb = spJ[c][jj];
            if (sa == sb || sa < 0 || sb < 0) continue;
            float x1, x2;
            if (table) {
                x1 = c1f[sa * g.S + sb];
                x2 = c2f[sa * g.S + sb];
            } else {
                const double d = __dsub_rn(g.z[sb], g.z[sa]);
                x1 = (float)__dmul_rn(2.0, d);
                x2 = (float)__dmul_rn(d, d);
            }
            const float pa = pfI[c][ii], pb = pfJ[c][jj], ja = dfI[ii], jb = dfJ[jj], j2 = Jf[ii][jj];
            const float v = __fadd_rn(__fmul_rn(x1, __fsub_rn(pa, pb)), __fmul_rn(x2, __fsub_rn(__fadd_rn(ja, jb), j2)));
            const float mag = fabsf(x1) * (fabsf(pa) + fabsf(pb)) + fabsf(x2) * (fabsf(ja) + fabsf(jb) + fabsf(j2));
            const float e = 1.9073486e-6f * mag + 9.5367432e-7f * fabsf(v) + 1e-30f;   // 2^-19, 2^-20
            lo[u] = v - e;
            ub = fminf(ub, v + e);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o; o >>= 1) ub = fminf(ub, __shfl_xor_sync(0xffffffffu, ub, o));
        if (lane == 0) redf[wid] = ub;
        if (threadIdx.x == 0) {
            tn = 0;
            tover = 0;
        }
        __syncthreads();
        float U = redf[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) U = fminf(U, redf[w]);
        const float thr = U + (float)kTie + 9.5367432e-7f * fabsf(U);
        // the candidates, in FP64 as the definition rounds them; a thread keeps its lowest two
        double cmin = INFINITY, v1 = INFINITY, v2 = INFINITY;
        unsigned long long k1 = ~0ull, k2 = ~0ull;
        int ncand = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (!(lo[u] <= thr)) continue;         // no pair: INFINITY (U is finite when a pair exists)
            const int jj = jq + u;
            const int sb = spJ[c][jj];
            double x1, x2;
            if (table) {
                x1 = c1t[sa * g.S + sb];
                x2 = c2t[sa * g.S + sb];
            } else {
                const double d = __dsub_rn(g.z[sb], g.z[sa]);
                x1 = __dmul_rn(2.0, d);
                x2 = __dmul_rn(d, d);
            }
            const double jab2 = 2.0 * g.J[(long)a * g.ld + j0 + jj];
            const double v = pair_dE_c(x1, x2, phI[c][ii], phJ[c][jj], dgI[ii], dgJ[jj], jab2);
            const unsigned long long k = (unsigned long long)a * (unsigned long long)g.Nv + (unsigned long long)(j0 + jj);
            ++ncand;
            cmin = fmin(cmin, v);
            if (v < v1) {
                v2 = v1;
                k2 = k1;
                v1 = v;
                k1 = k;
            } else if (v < v2) {
                v2 = v;
                k2 = k;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) cmin = fmin(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
        if (lane == 0) redv[wid] = cmin;
        __syncthreads();
        double tmin = redv[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) tmin = fmin(tmin, redv[w]);
        const double tlim = tmin + kTie;             // the tile's exact minimum + the tie
        if (ncand > 2 && v2 <= tlim) atomicOr(&tover, 1);   // a third could be in the tie set too
        if (v1 <= tlim) {
            const int slot = atomicAdd(&tn, 1);
            if (slot < GK) {
                tv[slot] = v1;
                tk[slot] = k1;
            }
        }
        if (v2 <= tlim) {
            const int slot = atomicAdd(&tn, 1);
            if (slot < GK) {
                tv[slot] = v2;
                tk[slot] = k2;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const long o = (long)blockIdx.x * g.B + b;
            g.cand_val[o] = tmin;
            g.tie_n[o] = tover ? GK + 1 : tn;
            for (int k = 0; k < GK && k < tn; ++k) {
                g.tie_val[o * GK + k] = tv[k];
                g.tie_key[o * GK + k] = tk[k];
            }
        }
        __syncthreads();
    }
}

// Pass 1, for the configurations whose relevant tie set overflowed: every
// pair in FP64 with the definition's roundings; per tile the lowest pair key
// (a Nv + b) with dE <= dmin + 1e-9 eV.
__global__ void __launch_bounds__(256) k_gd_pass1(GdArgs g)
{
    __shared__ double Jt[GT][GT + 1];
    __shared__ double phI[GD_CFG][GT], phJ[GD_CFG][GT];
    __shared__ int8_t spI[GD_CFG][GT], spJ[GD_CFG][GT];
    __shared__ int clI[GT], clJ[GT];
    __shared__ double dgI[GT], dgJ[GT];
    __shared__ double c1t[GS * GS], c2t[GS * GS];
    __shared__ unsigned long long redk[256];
    const int c0 = blockIdx.y * GD_CFG;
    bool any = false;
    for (int c = 0; c < GD_CFG; ++c) any |= c0 + c < g.B && g.active[c0 + c] && g.need1[c0 + c];
    if (!any) return;           // uniform over the block
    int bi, bj;
    gd_tile(blockIdx.x, bi, bj);
    const int i0 = bi * GT, j0 = bj * GT;
    for (int e = threadIdx.x; e < GT * GT; e += 256) {
        const int r = e / GT, c = e % GT;
        Jt[r][c] = 2.0 * g.J[(long)(i0 + r) * g.ld + j0 + c];    // exact
    }
    const bool table = g.S <= GS;
    if (table)
        for (int e = threadIdx.x; e < g.S * g.S; e += 256) {
            const double d = __dsub_rn(g.z[e % g.S], g.z[e / g.S]);     // [sa][sb]: z_sb - z_sa
            c1t[e] = __dmul_rn(2.0, d);
            c2t[e] = __dmul_rn(d, d);
        }
    for (int e = threadIdx.x; e < GT; e += 256) {
        const bool vi = i0 + e < g.Nv, vj = j0 + e < g.Nv;
        clI[e] = vi ? g.vclass[i0 + e] : -1;
        clJ[e] = vj ? g.vclass[j0 + e] : -2;
        dgI[e] = vi ? g.diag[i0 + e] : 0.0;
        dgJ[e] = vj ? g.diag[j0 + e] : 0.0;
    }
    for (int e = threadIdx.x; e < GD_CFG * GT; e += 256) {
        const int c = e / GT, x = e % GT, b = c0 + c;
        const bool okb = b < g.B;
        phI[c][x] = okb && i0 + x < g.Nv ? g.phi[(long)b * g.Nv + i0 + x] : 0.0;
        phJ[c][x] = okb && j0 + x < g.Nv ? g.phi[(long)b * g.Nv + j0 + x] : 0.0;
        spI[c][x] = okb && i0 + x < g.Nv ? g.species[(long)b * g.Nv + i0 + x] : (int8_t)-1;
        spJ[c][x] = okb && j0 + x < g.Nv ? g.species[(long)b * g.Nv + j0 + x] : (int8_t)-1;
    }
    __syncthreads();
    const int ii = threadIdx.x % GT;
    const int jq = (threadIdx.x / GT) * 16;
    for (int c = 0; c < GD_CFG; ++c) {
        const int b = c0 + c;
        const bool live = b < g.B && g.active[b] && g.need1[b];   // uniform over the block
        if (!live) continue;
        const double lim = g.dmin[b] + kTie;
        unsigned long long key = ~0ull;
        const int a = i0 + ii;
        const int sa = spI[c][ii];
        for (int jj = jq; jj < jq + 16; ++jj) {
            const int bb = j0 + jj;
            if (!(a < bb) || clI[ii] != clJ[jj]) continue;
            const int sb = spJ[c][jj];
            if (sa == sb || sa < 0 || sb < 0) continue;
            double x1, x2;
            if (table) {
                x1 = c1t[sa * g.S + sb];
                x2 = c2t[sa * g.S + sb];
            } else {
                const double d = __dsub_rn(g.z[sb], g.z[sa]);
                x1 = __dmul_rn(2.0, d);
                x2 = __dmul_rn(d, d);
            }
            const double dE = pair_dE_c(x1, x2, phI[c][ii], phJ[c][jj], dgI[ii], dgJ[jj], Jt[ii][jj]);
            if (dE <= lim) {
                const unsigned long long k = (unsigned long long)a * (unsigned long long)g.Nv + (unsigned long long)bb;
                if (k < key) key = k;
            }
        }
        redk[threadIdx.x] = key;
        __syncthreads();
        for (int w = 128; w; w >>= 1) {
            if (threadIdx.x < w) redk[threadIdx.x] = min(redk[threadIdx.x], redk[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) g.cand_key[(long)blockIdx.x * g.B + b] = redk[0];
        __syncthreads();
    }
}

// One warp per configuration: reduce the tile candidates; pass 0 retires
// configurations at a local minimum, pass 1 applies the chosen swap.
template <int PASS>
__global__ void k_gd_apply(GdArgs g, const double* __restrict__ Jfull, int8_t* __restrict__ species,
                           double* __restrict__ phi, int* __restrict__ active, double* __restrict__ dmin,
                           double* __restrict__ E, long long* __restrict__ steps, int* __restrict__ n_active,
                           int* __restrict__ need1, unsigned long long* __restrict__ chosen)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= g.B || !active[b]) return;
    if (PASS == 0) {
        double m = INFINITY;
        for (int t = lane; t < g.ntiles; t += 32) m = fmin(m, g.cand_val[(long)t * g.B + b]);
        for (int o = 16; o; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        // the lowest eligible pair from the tie sets of the tiles whose minimum is within kTie of m
        const double lim = m + kTie;
        unsigned long long k = ~0ull;
        int over = 0;
        for (int t = lane; t < g.ntiles; t += 32) {
            const long o = (long)t * g.B + b;
            if (!(g.cand_val[o] <= lim)) continue;
            const int n = g.tie_n[o];
            if (n > GK) over = 1;
            for (int e = 0; e < GK && e < n; ++e)
                if (g.tie_val[o * GK + e] <= lim) k = min(k, g.tie_key[o * GK + e]);
        }
        for (int o = 16; o; o >>= 1) {
            k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
            over |= __shfl_xor_sync(0xffffffffu, over, o);
        }
        if (lane == 0) {
            dmin[b] = m;
            need1[b] = over;
            chosen[b] = k;
            if (!(m < -kTie)) active[b] = 0;
            else atomicAdd(n_active, 1);
        }
        return;
    }
    unsigned long long k = chosen[b];
    if (need1[b]) {
        k = ~0ull;
        for (int t = lane; t < g.ntiles; t += 32) k = min(k, g.cand_key[(long)t * g.B + b]);
        for (int o = 16; o; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
    }
    const int a = (int)(k / (unsigned long long)g.Nv), c = (int)(k % (unsigned long long)g.Nv);
    int8_t* sp = species + (long)b * g.Nv;
    double* ph = phi + (long)b * g.Nv;
    const int sa = sp[a], sc = sp[c];
    const double d = __dsub_rn(g.z[sc], g.z[sa]);
    const double dE = pair_dE(d, ph[a], ph[c], g.diag[a], g.diag[c], Jfull[(long)a * g.ld + c]);
    __syncwarp();
    const double* ra = Jfull + (long)a * g.ld;
    const double* rc = Jfull + (long)c * g.ld;
    float* pf = g.phif + (long)b * g.Nv;
    for (int w = lane; w < g.Nv; w += 32) {
        const double v = __dadd_rn(ph[w], __dmul_rn(d, __dsub_rn(ra[w], rc[w])));
        ph[w] = v;
        pf[w] = (float)v;
    }
    __syncwarp();
    if (lane == 0) {
        sp[a] = (int8_t)sc;
        sp[c] = (int8_t)sa;
        E[b] = E[b] + dE;
        steps[b] += 1;
    }
}

__global__ void k_gd_init(int B, int* active, long long* steps)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        active[b] = 1;
        steps[b] = 0;
    }
}

}  // namespace

extern "C" goac_status goac_gd_run(goac_problem* p, int8_t* species_dev, int32_t B, int32_t max_steps,
                                   double* E_dev, int64_t* steps_dev)
{
    if (!p || B < 0 || B > GOAC_MAX_BATCH || max_steps < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_gd_run: bad argument");
    if (B == 0) return GOAC_OK;
    if (!species_dev || !E_dev || !steps_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_gd_run: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    goac_ctx* ctx = p->ctx;
    cudaStream_t st = ctx->stream;
    const int nb = (p->Nv + GT - 1) / GT;
    const int ntiles = nb * (nb + 1) / 2;
    const size_t tiles_b = (size_t)ntiles * B;
    const size_t nJ = (size_t)p->Nv_pad * p->Nv_pad;
    const size_t need = sizeof(double) * (size_t)B * p->Nv + sizeof(double) * tiles_b +
                        sizeof(unsigned long long) * tiles_b + sizeof(double) * tiles_b * GK +
                        sizeof(unsigned long long) * tiles_b * GK + sizeof(unsigned long long) * B +
                        sizeof(double) * B + sizeof(int) * (tiles_b + 2 * (size_t)B + 4) +
                        sizeof(float) * (nJ + (size_t)p->Nv + (size_t)B * p->Nv) + 4096;
    goac_status rc = goac::ensure(p->grad_tmp, need);
    if (rc) return rc;
    double* phi = (double*)p->grad_tmp.ptr;
    double* cval = phi + (size_t)B * p->Nv;
    unsigned long long* ckey = (unsigned long long*)(cval + tiles_b);
    double* tval = (double*)(ckey + tiles_b);
    unsigned long long* tkey = (unsigned long long*)(tval + tiles_b * GK);
    unsigned long long* chosen = tkey + tiles_b * GK;
    double* dmin = (double*)(chosen + B);
    int* active = (int*)(dmin + B);
    int* n_active = active + B;
    int* need1 = n_active + 4;
    int* tn = need1 + B;
    float* J2f = (float*)(((uintptr_t)(tn + tiles_b) + 255) & ~(uintptr_t)255);
    float* diagf = J2f + nJ;
    float* phif = diagf + p->Nv;
    // starting potentials: exact integer-digit contraction on the tensor cores
    // when the charges admit it, else the FP64 GEMM
    rc = goac::exact_supported(p) ? goac::phi_exact(p, species_dev, B, E_dev, phi)
                                  : goac::score_f64(p, species_dev, B, E_dev, phi);
    if (rc) return rc;
    goac::launch(k_gd_init, (B + 255) / 256, 256, 0, st, B, active, (long long*)steps_dev);
    goac::launch(k_gd_f32_consts, (int)std::min<size_t>((nJ + 255) / 256, 65535 * 4), 256, 0, st,
                 (const double*)p->J_vv, (long)nJ, (const double*)p->diag, p->Nv, J2f, diagf);
    goac::launch(k_gd_f32_phi, (int)std::min<size_t>(((size_t)B * p->Nv + 255) / 256, 65535 * 4), 256, 0, st,
                 (const double*)phi, (long)B * p->Nv, phif);
    GdArgs g;
    g.J = p->J_vv;
    g.diag = p->diag;
    g.species = species_dev;
    g.phi = phi;
    g.vclass = p->vclass_dev;
    g.z = p->z_dev;
    g.active = active;
    g.dmin = dmin;
    g.need1 = need1;
    g.cand_val = cval;
    g.cand_key = ckey;
    g.tie_val = tval;
    g.tie_key = tkey;
    g.tie_n = tn;
    g.J2f = J2f;
    g.diagf = diagf;
    g.phif = phif;
    g.ld = p->Nv_pad;
    g.Nv = p->Nv;
    g.B = B;
    g.ntiles = ntiles;
    g.S = p->S;
    dim3 grid(ntiles, (B + GD_CFG - 1) / GD_CFG);
    const int ablocks = (B + 7) / 8;
    for (int s = 0; s < max_steps; ++s) {
        GOAC_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), st));
        goac::launch(k_gd_pass0, grid, 256, 0, st, g);
        goac::launch(k_gd_apply<0>, ablocks, 256, 0, st, g, (const double*)p->J_vv, species_dev, phi, active, dmin,
                     E_dev, (long long*)steps_dev, n_active, need1, chosen);
        goac::launch(k_gd_pass1, grid, 256, 0, st, g);         // blocks without an overflowed tie set return
        goac::launch(k_gd_apply<1>, ablocks, 256, 0, st, g, (const double*)p->J_vv, species_dev, phi, active, dmin,
                     E_dev, (long long*)steps_dev, n_active, need1, chosen);
        GOAC_LAUNCH_CHECK("gd step");
        if ((s & 7) == 7 || s + 1 == max_steps) {
            int h = 0;
            GOAC_CUDA(cudaMemcpyAsync(&h, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
            GOAC_CUDA(cudaStreamSynchronize(st));
            if (h == 0) break;
        }
    }
    return GOAC_OK;
}
