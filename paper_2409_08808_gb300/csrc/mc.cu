// Parallel-chain Metropolis swap Monte Carlo (SI, Monte Carlo: neighbours
// differ by one atom swap; accept with P = min[1, exp(-dE/kT)]), for one
// problem (goac_mc_run) and for a batch of independent problems in one
// persistent launch with a device work queue (goac_batch_mc_run).
//
// One chain per warp.  The chain's potential phi = J q (over all sites, so
// including the fixed ions) and its species live in shared memory.  Proposals
// do not depend on the state (a uniformly random ordered pair of positions in
// a class), so each batch of 32 consecutive steps is drawn by the 32 lanes at
// once (Philox + the J_ab / diagonal gathers in parallel).  The batch is then
// evaluated speculatively: every pending lane computes its dE against the
// current state, a ballot finds the earliest accepting step, that step is
// committed (species swap, phi += d (J_a: - J_b:) with the warp reading the two
// J rows coalesced, E += dE), and the lanes after it are re-evaluated.  The
// result is exactly the sequential chain: steps before the first acceptance
// were evaluated against the same state they would have seen.
//
// The FP64 path uses explicitly rounded operations in the order of the
// definition (dE without contraction, the phi update as one fused multiply-add,
// acceptance as dE < -kT ln u), so its trajectory follows the FP64 definition
// step for step.  The FP32 path keeps J rows and phi in FP32.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

// Energy changes within 1e-9 eV of zero are treated as zero: swaps related by
// symmetry have dE = 0 exactly but +-1e-14 eV after rounding.
constexpr double kDeZero = 1e-9;

struct McProb {
    const void* J;            // Nv_pad x ld, R
    const void* diag;         // Nv, R
    const double* z;          // S
    const double* phifix;     // Nv
    const int32_t* cls_start; // ncls + 1
    const int32_t* cls_pos;   // Nv
    const uint32_t* wprefix;  // ncls
    int8_t* species;          // chains x Nv (in/out)
    const double* kT;         // chains (start temperature of an annealing schedule)
    const double* kT1;        // chains, end temperature of the schedule, or null (constant kT)
    int64_t total;            // schedule length in steps
    double* E_out;            // chains
    double* bestE;            // chains
    int8_t* best_species;     // chains x Nv or null
    int64_t* n_accept;        // chains or null
    int64_t* n_noop;          // chains or null: proposals of two positions with the same species
    int64_t* best_step;       // chains or null: step of the first visit of the best E (step0 - 1: start)
    int64_t* steps_done;      // chains or null: steps run
    int64_t patience;         // stop a chain after this many steps without improvement (0: never)
    double E_const;
    uint64_t seed;
    uint32_t wtotal;
    int ld, Nv, S, ncls, nmovable, only_movable, chains;
};

struct McScalars {
    int64_t n_steps;
    uint64_t step0;
};

template <typename R>
__device__ __forceinline__ R rd_add(R a, R b);
template <>
__device__ __forceinline__ double rd_add<double>(double a, double b) { return __dadd_rn(a, b); }
template <>
__device__ __forceinline__ float rd_add<float>(float a, float b) { return __fadd_rn(a, b); }
template <typename R>
__device__ __forceinline__ R rd_sub(R a, R b);
template <>
__device__ __forceinline__ double rd_sub<double>(double a, double b) { return __dsub_rn(a, b); }
template <>
__device__ __forceinline__ float rd_sub<float>(float a, float b) { return __fsub_rn(a, b); }
template <typename R>
__device__ __forceinline__ R rd_mul(R a, R b);
template <>
__device__ __forceinline__ double rd_mul<double>(double a, double b) { return __dmul_rn(a, b); }
template <>
__device__ __forceinline__ float rd_mul<float>(float a, float b) { return __fmul_rn(a, b); }

template <typename R>
__device__ __forceinline__ R rd_fma(R a, R b, R c);
template <>
__device__ __forceinline__ double rd_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float rd_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
};
template <>
struct Vec16<double> {
    using T = double2;
};

// Barrier over the W warps of one chain group (named barrier `id`, 1..15).
template <int W>
__device__ __forceinline__ void chain_sync(int id)
{
    if (W == 1) __syncwarp();
    else goacd::named_bar_sync(id, 32 * W);
}

// Run one chain with a group of W warps.  sp / phi point to the group's
// shared-memory slot.  All W warps draw and evaluate the same proposals (the
// decisions are identical), each updates its own slice of phi on acceptance,
// and the group synchronises after every acceptance.  phi_init / E_init: the
// chain's potential (J_vv q + phi_fix) and energy computed beforehand; when
// null (W == 1 only) the warp builds them itself.
template <typename R, int W>
__device__ void run_chain(const McProb& P, int chain, const McScalars& sc, int8_t* sp, R* phi,
                          const R* __restrict__ phi_init, const double* __restrict__ E_init, int bar_id)
{
    const int lane = threadIdx.x & 31;
    const int ct = threadIdx.x % (32 * W);     // thread index within the chain group
    const int cw = ct >> 5;                    // warp index within the chain group
    const int Nv = P.Nv, ld = P.ld;
    const R* J = (const R*)P.J;
    const R* diag = (const R*)P.diag;
    int8_t* gsp = P.species + (long)chain * Nv;

    double E;
    if (phi_init) {
        for (int w = ct; w < Nv; w += 32 * W) {
            sp[w] = gsp[w];
            phi[w] = phi_init[(long)chain * Nv + w];
        }
        E = E_init[chain];
        chain_sync<W>(bar_id);
    } else {
        // one warp: phi = J_vv q + phi_fix (rows of J read coalesced: J symmetric)
        for (int w = lane; w < Nv; w += 32) {
            sp[w] = gsp[w];
            phi[w] = (R)0;
        }
        __syncwarp();
        for (int w = 0; w < Nv; ++w) {
            const R qw = (R)P.z[sp[w]];
            if (qw == (R)0) continue;
            const R* row = J + (long)w * ld;
            for (int v = lane; v < Nv; v += 32) phi[v] = fma(row[v], qw, phi[v]);
        }
        __syncwarp();
        double e_part = 0.0;
        for (int v = lane; v < Nv; v += 32) {
            const double pf = P.phifix[v];
            phi[v] = (R)((double)phi[v] + pf);
            e_part += P.z[sp[v]] * ((double)phi[v] + pf);
        }
        for (int o = 16; o; o >>= 1) e_part += __shfl_xor_sync(0xffffffffu, e_part, o);
        E = e_part + P.E_const;
        __syncwarp();
    }
    double best = E;
    long nacc = 0, nnoop = 0;
    if (P.best_species)
        for (int w = ct; w < Nv; w += 32 * W) P.best_species[(long)chain * Nv + w] = sp[w];
    // run-level stop (no improvement for `patience` steps): steps t < t_stop run;
    // an acceptance that lowers E by more than 1e-9 eV below E_imp moves t_stop on
    const int64_t t_end = (int64_t)sc.step0 + sc.n_steps;
    int64_t t_best = (int64_t)sc.step0 - 1, t_imp = (int64_t)sc.step0 - 1;
    double E_imp = E;
    int64_t t_stop = P.patience > 0 ? min(t_end, t_imp + P.patience + 1) : t_end;

    const double kT = P.kT[chain];
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    // ---- this lane's proposal of the batch starting at step offset s0 (state independent) ----
    // The gathers diag[va], diag[vb], J[va][vb] are kept raw, so that the next batch's proposals
    // can be drawn and their loads issued before the current batch is evaluated.
    struct Prop {
        int va, vb;
        R da, db, jab;
        R thr;                     // accept iff dE <= 1e-9 eV or dE < thr = -kT ln u
    };
    auto draw = [&](int64_t s0, Prop& pr) {
        const int nb = (int)((sc.n_steps - s0) < 32 ? (sc.n_steps - s0) : 32);
        const uint64_t t = sc.step0 + (uint64_t)s0 + (uint64_t)lane;
        pr.va = pr.vb = 0;
        pr.da = pr.db = pr.jab = (R)0;
        pr.thr = (R)-INFINITY;
        if (lane < nb) {
            double kTl = kT;
            if (P.kT1 && P.total > 1)     // simulated annealing: kT0 (kT1/kT0)^(t/(total-1))
                kTl = kT * exp(log(P.kT1[chain] / kT) * ((double)t / (double)(P.total - 1)));
            const uint4 x = goacd::philox(make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)chain, 0u), k0, k1);
            int k = P.only_movable;
            if (P.nmovable != 1) {
                const uint4 y =
                    goacd::philox(make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)chain, 1u), k0, k1);
                const uint32_t th = goacd::draw_below(y.x, P.wtotal);
                k = P.ncls - 1;
                for (int c = 0; c < P.ncls; ++c)
                    if (P.wprefix[c] > th) {
                        k = c;
                        break;
                    }
            }
            const int start = P.cls_start[k];
            const uint32_t n = (uint32_t)(P.cls_start[k + 1] - start);
            const uint32_t a = goacd::draw_below(x.x, n);
            const uint32_t bb = goacd::draw_below(x.y, n - 1);
            const uint32_t b = bb + (bb >= a);
            pr.va = P.cls_pos[start + a];
            pr.vb = P.cls_pos[start + b];
            const double u = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6)) * (1.0 / 9007199254740992.0);
            pr.da = diag[pr.va];
            pr.db = diag[pr.vb];
            pr.jab = J[(long)pr.va * ld + pr.vb];
            // Metropolis: u < exp(-dE/kT) is the event dE < -kT ln u, so the
            // threshold is formed once per proposal, not per evaluation
            if (kTl > 0.0) {
                if (u == 0.0) pr.thr = (R)INFINITY;
                else if (sizeof(R) == 8) pr.thr = (R)(-kTl * log(u));
                else pr.thr = (R)(-(float)kTl * logf((float)u));
            }
        }
    };
    Prop cur, nxt;
    if (W > 1 && sc.n_steps > 0) draw(0, nxt);
    for (int64_t s0 = 0; s0 < sc.n_steps; s0 += 32) {
        const int64_t tb = (int64_t)sc.step0 + s0;      // first step of this batch
        if (tb >= t_stop) break;
        const int nb = (int)((sc.n_steps - s0) < 32 ? (sc.n_steps - s0) : 32);
        if (W > 1) {                                     // the next batch's loads fly meanwhile
            cur = nxt;
            if (s0 + 32 < sc.n_steps) draw(s0 + 32, nxt);
        } else {
            draw(s0, cur);
        }
        const int va = cur.va, vb = cur.vb;
        const R thr = cur.thr;
        const R jsum = rd_sub<R>(rd_add<R>(cur.da, cur.db), rd_mul<R>((R)2, cur.jab));
        const uint32_t valid = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
        // lanes whose step lies before t_stop
        auto live = [&](int64_t ts) -> uint32_t {
            const int64_t k = ts - tb;
            return k >= 32 ? 0xffffffffu : (k <= 0 ? 0u : ((1u << k) - 1u));
        };
        uint32_t pending = valid & live(t_stop);
        while (pending) {
            bool acc = false, noop = false;
            R d = (R)0, dE = (R)0;
            if ((pending >> lane) & 1u) {
                const int sa = sp[va], sb = sp[vb];
                noop = sa == sb;
                if (sa != sb) {
                    d = (R)(P.z[sb] - P.z[sa]);
                    dE = rd_add<R>(rd_mul<R>(rd_mul<R>((R)2, d), rd_sub<R>(phi[va], phi[vb])),
                                   rd_mul<R>(rd_mul<R>(d, d), jsum));
                    acc = (double)dE <= kDeZero || dE < thr;
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, acc);
            const uint32_t nm = __ballot_sync(0xffffffffu, noop);
            if (m == 0u) {                         // every pending step is rejected or a no-op
                nnoop += __popc(nm);
                break;
            }
            const int kl = __ffs(m) - 1;
            nnoop += __popc(nm & ((1u << kl) - 1u));   // steps before the acceptance are final
            const int ca = __shfl_sync(0xffffffffu, va, kl);
            const int cb = __shfl_sync(0xffffffffu, vb, kl);
            const R cd = __shfl_sync(0xffffffffu, d, kl);
            const R cdE = __shfl_sync(0xffffffffu, dE, kl);
            chain_sync<W>(bar_id);                 // every warp has read the state it evaluated
            if (ct == 0) {
                const int8_t ta = sp[ca];
                sp[ca] = sp[cb];
                sp[cb] = ta;
            }
            if (cd != (R)0 && W == 1) {
                const R* __restrict__ ra = J + (long)ca * ld;
                const R* __restrict__ rb = J + (long)cb * ld;
                // one warp: 8 loads of each row in flight per lane
                for (int w0 = lane; w0 < Nv; w0 += 32 * 8) {
                    R xa[8], xb[8];
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu) {
                        const int w = w0 + 32 * uu;
                        xa[uu] = w < Nv ? ra[w] : (R)0;
                        xb[uu] = w < Nv ? rb[w] : (R)0;
                    }
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu) {
                        const int w = w0 + 32 * uu;
                        if (w < Nv) phi[w] = rd_fma<R>(cd, rd_sub<R>(xa[uu], xb[uu]), phi[w]);
                    }
                }
            } else if (cd != (R)0) {
                const R* __restrict__ ra = J + (long)ca * ld;
                const R* __restrict__ rb = J + (long)cb * ld;
                // W warps: 16-byte vectors of both rows (rows are ld >= Nv long, ld a multiple of 128), U
                // of each in flight per thread; phi (its slot rounded up to 16 bytes) read and written as
                // vectors, each element updated as phi + d (J_a - J_b) exactly as one element at a time
                constexpr int V = 16 / (int)sizeof(R);
                constexpr int U = 4;
                using VT = typename Vec16<R>::T;
                for (int w0 = ct * V; w0 < Nv; w0 += 32 * W * V * U) {
                    VT xa[U], xb[U];
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                        const int w = w0 + 32 * W * V * uu;
                        if (w < Nv) {
                            xa[uu] = *reinterpret_cast<const VT*>(ra + w);
                            xb[uu] = *reinterpret_cast<const VT*>(rb + w);
                        }
                    }
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                        const int w = w0 + 32 * W * V * uu;
                        if (w < Nv) {
                            VT pv = *reinterpret_cast<const VT*>(phi + w);
                            R* pe = reinterpret_cast<R*>(&pv);
                            const R* ae = reinterpret_cast<const R*>(&xa[uu]);
                            const R* be = reinterpret_cast<const R*>(&xb[uu]);
#pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (w + e < Nv) pe[e] = rd_fma<R>(cd, rd_sub<R>(ae[e], be[e]), pe[e]);
                            *reinterpret_cast<VT*>(phi + w) = pv;
                        }
                    }
                }
            }
            chain_sync<W>(bar_id);
            E = E + (double)cdE;
            ++nacc;
            if (E < best - kDeZero) {          // a new best: lower by more than the tie
                best = E;
                t_best = tb + kl;
                if (P.best_species) {
                    for (int w = ct; w < Nv; w += 32 * W) P.best_species[(long)chain * Nv + w] = sp[w];
                    chain_sync<W>(bar_id);
                }
            }
            if (P.patience > 0 && E < E_imp - kDeZero) {
                E_imp = E;
                t_imp = tb + kl;
                t_stop = min(t_end, t_imp + P.patience + 1);
            }
            // the steps after the committed one, up to t_stop (which an improvement moves on)
            pending = valid & ~((2u << kl) - 1u) & live(t_stop);
        }
    }
    chain_sync<W>(bar_id);
    for (int w = ct; w < Nv; w += 32 * W) gsp[w] = sp[w];
    if (ct == 0) {
        P.E_out[chain] = E;
        P.bestE[chain] = best;
        if (P.n_accept) P.n_accept[chain] = nacc;
        if (P.n_noop) P.n_noop[chain] = nnoop;
        if (P.best_step) P.best_step[chain] = t_best;
        if (P.steps_done) P.steps_done[chain] = t_stop - (int64_t)sc.step0;
    }
}

__host__ __device__ inline size_t warp_slot_bytes(int Nv, int rbytes)
{
    size_t a = ((size_t)Nv * rbytes + 15) & ~(size_t)15;
    size_t b = ((size_t)Nv + 15) & ~(size_t)15;
    return a + b;
}

// Single problem: W warps per chain, chains_per_cta chains per CTA, phi / E
// initialised beforehand by the scoring GEMM.
template <typename R, int W>
__global__ void k_mc(McProb P, McScalars sc, const R* __restrict__ phi_init, const double* __restrict__ E_init,
                     int* err)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int slot_i = threadIdx.x / (32 * W);
    const int chain = blockIdx.x * (blockDim.x / (32 * W)) + slot_i;
    if (chain >= P.chains) return;     // whole chain groups leave together
    const size_t slot = warp_slot_bytes(P.Nv, sizeof(R));
    uint8_t* base = smem + slot * slot_i;
    R* phi = (R*)base;
    int8_t* sp = (int8_t*)(base + (((size_t)P.Nv * sizeof(R) + 15) & ~(size_t)15));
    run_chain<R, W>(P, chain, sc, sp, phi, phi_init, E_init, 1 + slot_i);
    (void)err;
}

// One warp per chain with the potential built in the kernel (the per-problem
// launches of the batched baseline use the same chain code as the persistent
// batched kernel).
template <typename R>
__global__ void k_mc_single(McProb P, McScalars sc, int* err)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int wib = threadIdx.x >> 5;
    const int chain = blockIdx.x * (blockDim.x >> 5) + wib;
    if (chain >= P.chains) return;
    const size_t slot = warp_slot_bytes(P.Nv, sizeof(R));
    uint8_t* base = smem + slot * wib;
    R* phi = (R*)base;
    int8_t* sp = (int8_t*)(base + (((size_t)P.Nv * sizeof(R) + 15) & ~(size_t)15));
    run_chain<R, 1>(P, chain, sc, sp, phi, nullptr, nullptr, 0);
    (void)err;
}

// Batch of problems: persistent warps take (problem, chain) items from a queue.
template <typename R>
__global__ void k_mc_batch(const McProb* __restrict__ probs, const int2* __restrict__ items, int n_items,
                           int* __restrict__ counter, const McScalars* __restrict__ scp, int max_nv, int* err)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const size_t slot = warp_slot_bytes(max_nv, sizeof(R));
    uint8_t* base = smem + slot * wib;
    const McScalars sc = *scp;
    while (true) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const int2 pc = items[it];
        const McProb P = probs[pc.x];
        R* phi = (R*)base;
        int8_t* sp = (int8_t*)(base + (((size_t)P.Nv * sizeof(R) + 15) & ~(size_t)15));
        run_chain<R, 1>(P, pc.y, sc, sp, phi, nullptr, nullptr, 0);
        __syncwarp();
    }
}

McProb make_desc(goac_problem* p, bool f32, int8_t* species, int C, const double* kT, double* E, double* bestE,
                 int8_t* best_species, int64_t* nacc, uint64_t seed)
{
    McProb d;
    d.J = f32 ? (const void*)p->J_f32 : (const void*)p->J_vv;
    d.diag = f32 ? (const void*)p->diag_f32 : (const void*)p->diag;
    d.z = p->z_dev;
    d.phifix = p->phifix;
    d.cls_start = p->cls_start_dev;
    d.cls_pos = p->cls_pos_dev;
    d.wprefix = p->wprefix_dev;
    d.species = species;
    d.kT = kT;
    d.kT1 = nullptr;
    d.total = 0;
    d.E_out = E;
    d.bestE = bestE;
    d.best_species = best_species;
    d.n_accept = nacc;
    d.n_noop = nullptr;
    d.best_step = nullptr;
    d.steps_done = nullptr;
    d.patience = 0;
    d.E_const = p->E_const;
    d.seed = seed;
    d.wtotal = p->wtotal;
    d.ld = p->Nv_pad;
    d.Nv = p->Nv;
    d.S = p->S;
    d.ncls = p->ncls;
    d.nmovable = p->nmovable;
    d.only_movable = p->only_movable;
    d.chains = C;
    return d;
}

constexpr size_t kSmemBudget = 220 * 1024;

// Most chains per CTA that k_mc<R, W> can launch with (its register count
// limits the threads of a block below 1,024 when it is above 64 per thread).
template <typename R, int W>
int mc_cpc_limit()
{
    static int lim = 0;
    if (!lim) {
        cudaFuncAttributes fa;
        const int mt = cudaFuncGetAttributes(&fa, k_mc<R, W>) == cudaSuccess ? fa.maxThreadsPerBlock : 1024;
        lim = std::max(1, mt / (32 * W));
    }
    return lim;
}

int mc_cpc_limit(bool f32, int W)
{
    if (f32) return W == 4 ? mc_cpc_limit<float, 4>() : W == 2 ? mc_cpc_limit<float, 2>() : mc_cpc_limit<float, 1>();
    return W == 4 ? mc_cpc_limit<double, 4>() : W == 2 ? mc_cpc_limit<double, 2>() : mc_cpc_limit<double, 1>();
}

}  // namespace

// W_force / cpc_force (> 0) override the launch shape (the autotuner's probes).
static goac_status mc_run_impl(goac_problem* p, int8_t* species_dev, int32_t C, const double* kT_dev,
                               const double* kT1_dev, int64_t total, int64_t n_steps, uint64_t seed, uint64_t step0,
                               int32_t precision, double* E_dev, double* bestE_dev, int8_t* best_species_dev,
                               int64_t* n_accept_dev, int W_force = 0, int cpc_force = 0, int64_t patience = 0,
                               const goac_mc_stats* stats = nullptr)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: NULL problem");
    if (C < 0 || C > GOAC_MAX_BATCH || n_steps < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: bad size");
    if (precision != GOAC_PREC_F64 && precision != GOAC_PREC_F32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: precision must be F64 or F32");
    if (p->nmovable == 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: no class has two positions");
    if (C == 0) return GOAC_OK;
    if (!species_dev || !kT_dev || !E_dev || !bestE_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const bool f32 = precision == GOAC_PREC_F32;
    if (f32) {
        goac_status rc = goac::prepare_f32(p);
        if (rc) return rc;
    }
    const size_t slot = warp_slot_bytes(p->Nv, f32 ? 4 : 8);
    if (slot > kSmemBudget)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run: Nv too large for a shared-memory chain");
    // potentials and energies of all chains
    const size_t rb = f32 ? 4 : 8;
    goac_status rc = goac::ensure(p->phi, rb * (size_t)C * p->Nv + sizeof(double) * (size_t)C + 256);
    if (rc) return rc;
    void* phi0 = p->phi.ptr;
    double* E0 = (double*)((char*)p->phi.ptr + ((rb * (size_t)C * p->Nv + 255) & ~(size_t)255));
    // (the exact integer-digit contraction on the tensor cores when the charges
    // admit it, phi rounded to FP32 once for FP32 chains; else the FP64 or FP32
    // CUDA-core GEMM)
    if (goac::exact_supported(p)) rc = goac::phi_exact(p, species_dev, C, E0, phi0, f32);
    else if (f32) rc = goac::score_f32(p, species_dev, C, E0, (float*)phi0);
    else rc = goac::score_f64(p, species_dev, C, E0, (double*)phi0);
    if (rc) return rc;
    // launch shape: warps per chain (more warps share the O(Nv) update of a long
    // chain) and chains per CTA, from the autotuner when it has run for this
    // problem and precision, else by size; the trajectories do not depend on it
    const int* tuned = p->mc_tuned[f32 ? 1 : 0];
    int W = W_force ? W_force : (tuned[0] ? tuned[0] : (p->Nv >= 3072 ? 4 : (p->Nv >= 1536 ? 2 : 1)));
    int cpc = (int)(kSmemBudget / slot);
    cpc = std::min(cpc, mc_cpc_limit(f32, W));
    cpc = std::min(cpc, cpc_force ? cpc_force : (tuned[1] ? tuned[1] : 15));
    cpc = std::min(cpc, C);
    if (cpc < 1) cpc = 1;
    const size_t smem = slot * cpc;
    McProb d = make_desc(p, f32, species_dev, C, kT_dev, E_dev, bestE_dev, best_species_dev, n_accept_dev, seed);
    d.kT1 = kT1_dev;
    d.total = total;
    d.patience = patience;
    if (stats) {
        if (stats->n_accept_dev) d.n_accept = stats->n_accept_dev;
        d.n_noop = stats->n_noop_dev;
        d.best_step = stats->best_step_dev;
        d.steps_done = stats->steps_dev;
    }
    McScalars sc{n_steps, step0};
    const int blocks = (C + cpc - 1) / cpc;
    goac::KTimer kt(p->ctx, goac::KID_MC, p->ctx->stream);
#define GOAC_MC_LAUNCH(RT, WW)                                                                                  \
    do {                                                                                                        \
        GOAC_CUDA(cudaFuncSetAttribute(k_mc<RT, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));  \
        goac::launch(k_mc<RT, WW>, blocks, 32 * WW * cpc, smem, p->ctx->stream, d, sc, (const RT*)phi0,           \
                     (const double*)E0, p->ctx->d_err);                                                         \
    } while (0)
    if (f32) {
        if (W == 4) GOAC_MC_LAUNCH(float, 4);
        else if (W == 2) GOAC_MC_LAUNCH(float, 2);
        else GOAC_MC_LAUNCH(float, 1);
    } else {
        if (W == 4) GOAC_MC_LAUNCH(double, 4);
        else if (W == 2) GOAC_MC_LAUNCH(double, 2);
        else GOAC_MC_LAUNCH(double, 1);
    }
#undef GOAC_MC_LAUNCH
    GOAC_LAUNCH_CHECK("k_mc");
    return GOAC_OK;
}

extern "C" goac_status goac_mc_run(goac_problem* p, int8_t* species_dev, int32_t C, const double* kT_dev,
                                   int64_t n_steps, uint64_t seed, uint64_t step0, int32_t precision, double* E_dev,
                                   double* bestE_dev, int8_t* best_species_dev, int64_t* n_accept_dev)
{
    return mc_run_impl(p, species_dev, C, kT_dev, nullptr, 0, n_steps, seed, step0, precision, E_dev, bestE_dev,
                       best_species_dev, n_accept_dev);
}

extern "C" goac_status goac_mc_run_ex(goac_problem* p, int8_t* species_dev, int32_t C, const double* kT_dev,
                                      int64_t n_steps, uint64_t seed, uint64_t step0, int32_t precision,
                                      int64_t patience, double* E_dev, double* bestE_dev, int8_t* best_species_dev,
                                      const goac_mc_stats* stats)
{
    if (patience < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_run_ex: patience must be >= 0");
    return mc_run_impl(p, species_dev, C, kT_dev, nullptr, 0, n_steps, seed, step0, precision, E_dev, bestE_dev,
                       best_species_dev, nullptr, 0, 0, patience, stats);
}

extern "C" goac_status goac_sa_run(goac_problem* p, int8_t* species_dev, int32_t C, const double* kT0_dev,
                                   const double* kT1_dev, int64_t total_steps, int64_t n_steps, uint64_t seed,
                                   uint64_t step0, int32_t precision, double* E_dev, double* bestE_dev,
                                   int8_t* best_species_dev, int64_t* n_accept_dev)
{
    if (total_steps < 1) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_sa_run: total_steps must be >= 1");
    if (C != 0 && !kT1_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_sa_run: kT1 needed");
    return mc_run_impl(p, species_dev, C, kT0_dev, kT1_dev, total_steps, n_steps, seed, step0, precision, E_dev,
                       bestE_dev, best_species_dev, n_accept_dev);
}

// Autotuner of the single-problem Monte Carlo launch: every (warps per chain,
// chains per CTA) in {1, 2, 4} x {1, 2, 4, 8, 15} that fits runs `probe_steps`
// steps on a scratch copy of the chains (twice, the second timed with CUDA
// events on the context stream); the fastest is kept for this problem and
// precision and used by later goac_mc_run / goac_sa_run / goac_remc_run calls.
extern "C" goac_status goac_mc_autotune(goac_problem* p, const int8_t* species_dev, int32_t C, const double* kT_dev,
                                        int64_t probe_steps, int32_t precision, int32_t* W_out, int32_t* cpc_out,
                                        double* ms_out)
{
    if (!p || !species_dev || !kT_dev || C <= 0 || C > GOAC_MAX_BATCH || probe_steps <= 0)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_autotune: bad argument");
    if (precision != GOAC_PREC_F64 && precision != GOAC_PREC_F32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_autotune: precision must be F64 or F32");
    if (p->nmovable == 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_autotune: no class has two positions");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    cudaStream_t st = p->ctx->stream;
    const size_t sp_bytes = ((size_t)C * p->Nv + 255) & ~(size_t)255;
    DevBuf scratch;
    goac_status rc = goac::ensure(scratch, sp_bytes + 2 * sizeof(double) * (size_t)C + 256);
    if (rc) return rc;
    int8_t* sp = (int8_t*)scratch.ptr;
    double* E = (double*)((char*)scratch.ptr + sp_bytes);
    double* bE = E + C;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int bestW = 0, bestc = 0;
    float best_t = 0.0f;
    const int Ws[3] = {1, 2, 4}, cpcs[5] = {1, 2, 4, 8, 15};
    const size_t slot = warp_slot_bytes(p->Nv, precision == GOAC_PREC_F32 ? 4 : 8);
    for (int wi = 0; wi < 3 && !rc; ++wi) {
        for (int ci = 0; ci < 5 && !rc; ++ci) {
            const int W = Ws[wi], cpc = cpcs[ci];
            if (slot * cpc > kSmemBudget || cpc > mc_cpc_limit(precision == GOAC_PREC_F32, W) ||
                (cpc > C && cpc != 1))
                continue;
            for (int rep = 0; rep < 2 && !rc; ++rep) {
                const cudaError_t e = cudaMemcpyAsync(sp, species_dev, (size_t)C * p->Nv, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) {
                    rc = goac::cuda_fail(e, "goac_mc_autotune: copy");
                    break;
                }
                if (rep == 1) cudaEventRecord(a, st);
                rc = mc_run_impl(p, sp, C, kT_dev, nullptr, 0, probe_steps, 12345u, 0, precision, E, bE, nullptr,
                                 nullptr, W, cpc);
                if (!rc && rep == 1) cudaEventRecord(b, st);
            }
            if (rc) break;
            cudaEventSynchronize(b);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (bestW == 0 || ms < best_t) {
                bestW = W;
                bestc = cpc;
                best_t = ms;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(st);
    cudaFree(scratch.ptr);
    if (rc) return rc;
    if (bestW == 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_autotune: no launch shape fits");
    int* tuned = p->mc_tuned[precision == GOAC_PREC_F32 ? 1 : 0];
    tuned[0] = bestW;
    tuned[1] = bestc;
    if (W_out) *W_out = bestW;
    if (cpc_out) *cpc_out = bestc;
    if (ms_out) *ms_out = best_t;
    return GOAC_OK;
}

// Fix the Monte Carlo launch shape of a problem (no counterpart in the paper):
// what goac_mc_autotune would store, set by the caller; 0 restores the
// size-based choice.  The trajectories do not depend on it.
extern "C" goac_status goac_mc_set_shape(goac_problem* p, int32_t precision, int32_t W, int32_t chains_per_cta)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_set_shape: NULL problem");
    if (precision != GOAC_PREC_F64 && precision != GOAC_PREC_F32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_set_shape: precision must be F64 or F32");
    if (!(W == 0 || W == 1 || W == 2 || W == 4) || chains_per_cta < 0 || chains_per_cta > 32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_mc_set_shape: W must be 0, 1, 2 or 4 and chains per CTA 0..32");
    int* tuned = p->mc_tuned[precision == GOAC_PREC_F32 ? 1 : 0];
    tuned[0] = W;
    tuned[1] = chains_per_cta;
    return GOAC_OK;
}

namespace {

__global__ void k_remc_init(int G, int R, const double* __restrict__ ladder, double* __restrict__ kT,
                            int32_t* __restrict__ perm, unsigned long long* __restrict__ nex)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *nex = 0ull;
    if (c >= G * R) return;
    perm[c] = c;
    kT[c] = ladder[c % R];
}

// Exchange attempts after round r, one thread per replica group.
__global__ void k_remc_exchange(int G, int R, uint32_t r, const double* __restrict__ ladder, double* __restrict__ kT,
                                const double* __restrict__ E, int32_t* __restrict__ perm, uint64_t seed,
                                unsigned long long* __restrict__ nex)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    unsigned long long cnt = 0;
    for (int k = (int)(r & 1u); k + 1 < R; k += 2) {
        const int ca = perm[g * R + k], cb = perm[g * R + k + 1];
        const double dE = E[ca] - E[cb];
        const double x = dE * (1.0 / ladder[k] - 1.0 / ladder[k + 1]);
        const uint4 w = goacd::philox(make_uint4(r, (uint32_t)g, (uint32_t)k, 6u), k0, k1);
        const double u = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) * (1.0 / 9007199254740992.0);
        if (x >= 0.0 || u < exp(x)) {
            perm[g * R + k] = cb;
            perm[g * R + k + 1] = ca;
            kT[ca] = ladder[k + 1];
            kT[cb] = ladder[k];
            ++cnt;
        }
    }
    if (cnt) atomicAdd(nex, cnt);
}

}  // namespace

extern "C" goac_status goac_remc_run(goac_problem* p, int8_t* species_dev, int32_t G, int32_t R,
                                     const double* kT_ladder_host, int32_t n_rounds, int64_t steps_per_round,
                                     uint64_t seed, int32_t precision, double* E_dev, int32_t* perm_dev,
                                     int64_t* n_exchanges_host)
{
    if (!p || G < 0 || R <= 0 || n_rounds < 0 || steps_per_round < 0 || (int64_t)G * R > GOAC_MAX_BATCH)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_remc_run: bad argument");
    if (G == 0) {
        if (n_exchanges_host) *n_exchanges_host = 0;
        return GOAC_OK;
    }
    if (!species_dev || !kT_ladder_host || !E_dev || !perm_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_remc_run: NULL argument");
    for (int k = 0; k < R; ++k)
        if (!(kT_ladder_host[k] > 0.0)) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_remc_run: temperatures must be > 0");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const int C = G * R;
    DevBuf& buf = p->score_tmp;
    goac_status rc = goac::ensure(buf, sizeof(double) * (2 * (size_t)C + R) + 64);
    if (rc) return rc;
    double* kT = (double*)buf.ptr;
    double* bestE = kT + C;
    double* ladder = bestE + C;
    unsigned long long* nex = (unsigned long long*)(ladder + R);
    cudaStream_t st = p->ctx->stream;
    GOAC_CUDA(cudaMemcpyAsync(ladder, kT_ladder_host, sizeof(double) * R, cudaMemcpyHostToDevice, st));
    goac::launch(k_remc_init, (C + 255) / 256, 256, 0, st, G, R, (const double*)ladder, kT, perm_dev, nex);
    GOAC_LAUNCH_CHECK("k_remc_init");
    for (int r = 0; r < n_rounds; ++r) {
        rc = mc_run_impl(p, species_dev, C, kT, nullptr, 0, steps_per_round, seed, (uint64_t)r * steps_per_round,
                         precision, E_dev, bestE, nullptr, nullptr);
        if (rc) return rc;
        goac::launch(k_remc_exchange, (G + 127) / 128, 128, 0, st, G, R, (uint32_t)r, (const double*)ladder, kT,
                     (const double*)E_dev, perm_dev, seed, nex);
        GOAC_LAUNCH_CHECK("k_remc_exchange");
    }
    if (n_exchanges_host) {
        unsigned long long h = 0;
        GOAC_CUDA(cudaMemcpyAsync(&h, nex, sizeof(h), cudaMemcpyDeviceToHost, st));
        GOAC_CUDA(cudaStreamSynchronize(st));
        *n_exchanges_host = (int64_t)h;
    }
    return GOAC_OK;
}

extern "C" goac_status goac_batch_mc_run(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs,
                                         int8_t* const* species_dev, const int32_t* chains,
                                         const double* const* kT_dev, int64_t n_steps, uint64_t seed,
                                         uint64_t step0, int32_t precision, double* const* E_dev,
                                         double* const* bestE_dev, int32_t chains_per_cta, int32_t mode)
{
    if (!ctx || !probs || n_probs <= 0 || !species_dev || !chains || !kT_dev || !E_dev || !bestE_dev)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: bad argument");
    if (precision != GOAC_PREC_F64 && precision != GOAC_PREC_F32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: precision must be F64 or F32");
    if (mode < 0 || mode > 2) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: mode must be 0, 1 or 2");
    if (chains_per_cta < 1 || chains_per_cta > 32)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: chains_per_cta must be in [1, 32]");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    const bool f32 = precision == GOAC_PREC_F32;
    const int rb = f32 ? 4 : 8;
    std::vector<McProb> descs(n_probs);
    std::vector<int2> items;
    int max_nv = 0;
    uint64_t key = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    for (int i = 0; i < n_probs; ++i) {
        goac_problem* p = probs[i];
        if (!p || chains[i] < 0 || (chains[i] > 0 && (!species_dev[i] || !kT_dev[i] || !E_dev[i] || !bestE_dev[i])))
            return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: bad per-problem argument");
        if ((int64_t)items.size() + chains[i] > GOAC_MAX_BATCH)
            return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: more than GOAC_MAX_BATCH chains in all");
        if (p->ctx != ctx) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: problem from another context");
        if (p->nmovable == 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: problem without moves");
        if (f32) {
            goac_status rc = goac::prepare_f32(p);
            if (rc) return rc;
        }
        descs[i] = make_desc(p, f32, species_dev[i], chains[i], kT_dev[i], E_dev[i], bestE_dev[i], nullptr, nullptr,
                             seed + (uint64_t)i);
        for (int c = 0; c < chains[i]; ++c) items.push_back(make_int2(i, c));
        if (p->Nv > max_nv) max_nv = p->Nv;
        mix((uint64_t)(uintptr_t)p);
        mix((uint64_t)(uintptr_t)species_dev[i]);
        mix((uint64_t)(uintptr_t)kT_dev[i]);
        mix((uint64_t)(uintptr_t)E_dev[i]);
        mix((uint64_t)(uintptr_t)bestE_dev[i]);
        mix((uint64_t)chains[i]);
    }
    mix(seed);
    mix((uint64_t)precision);
    mix((uint64_t)chains_per_cta);
    const size_t slot = warp_slot_bytes(max_nv, rb);
    if (slot * chains_per_cta > kSmemBudget)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_run: chains_per_cta x largest cell exceeds shared memory");
    cudaStream_t st = ctx->stream;
    const int n_items = (int)items.size();
    if (n_items == 0) return GOAC_OK;

    if (mode == 0) {
        // baseline: one launch per problem
        McScalars sc{n_steps, step0};
        for (int i = 0; i < n_probs; ++i) {
            if (descs[i].chains == 0) continue;
            const size_t s1 = warp_slot_bytes(descs[i].Nv, rb);
            int wpb = chains_per_cta < descs[i].chains ? chains_per_cta : descs[i].chains;
            const size_t smem = s1 * wpb;
            const int blocks = (descs[i].chains + wpb - 1) / wpb;
            if (f32) {
                GOAC_CUDA(cudaFuncSetAttribute(k_mc_single<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmemBudget));
                goac::launch(k_mc_single<float>, blocks, 32 * wpb, smem, st, descs[i], sc, ctx->d_err);
            } else {
                GOAC_CUDA(cudaFuncSetAttribute(k_mc_single<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmemBudget));
                goac::launch(k_mc_single<double>, blocks, 32 * wpb, smem, st, descs[i], sc, ctx->d_err);
            }
            GOAC_LAUNCH_CHECK("k_mc (per problem)");
        }
        return GOAC_OK;
    }

    // persistent: descriptors, items, queue counter and per-call scalars on the device
    const size_t desc_bytes = sizeof(McProb) * n_probs;
    const size_t item_bytes = sizeof(int2) * n_items;
    goac_status rc = goac::ensure(ctx->batch_desc, desc_bytes);
    if (!rc) rc = goac::ensure(ctx->batch_items, item_bytes);
    if (!rc) rc = goac::ensure(ctx->batch_counter, 64);
    if (rc) return rc;
    const bool reuse = mode == 2 && ctx->batch_graph && ctx->batch_graph_key == key;
    McScalars sc{n_steps, step0};
    int* counter = (int*)ctx->batch_counter.ptr;
    McScalars* d_sc = (McScalars*)((char*)ctx->batch_counter.ptr + 16);
    if (!reuse) {
        GOAC_CUDA(cudaMemcpyAsync(ctx->batch_desc.ptr, descs.data(), desc_bytes, cudaMemcpyHostToDevice, st));
        GOAC_CUDA(cudaMemcpyAsync(ctx->batch_items.ptr, items.data(), item_bytes, cudaMemcpyHostToDevice, st));
    }
    GOAC_CUDA(cudaMemcpyAsync(d_sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
    const size_t smem = slot * chains_per_cta;
    int per_sm = 1;
    if (f32) {
        GOAC_CUDA(cudaFuncSetAttribute(k_mc_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GOAC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mc_batch<float>, 32 * chains_per_cta, smem));
    } else {
        GOAC_CUDA(cudaFuncSetAttribute(k_mc_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GOAC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mc_batch<double>, 32 * chains_per_cta, smem));
    }
    if (per_sm < 1) per_sm = 1;
    int grid = ctx->num_sms * per_sm;
    const int need = (n_items + chains_per_cta - 1) / chains_per_cta;
    if (grid > need) grid = need;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        if (f32)
            goac::launch(k_mc_batch<float>, grid, 32 * chains_per_cta, smem, st, (const McProb*)ctx->batch_desc.ptr,
                                                                        (const int2*)ctx->batch_items.ptr, n_items,
                                                                        counter, d_sc, max_nv, ctx->d_err);
        else
            goac::launch(k_mc_batch<double>, grid, 32 * chains_per_cta, smem, st, (const McProb*)ctx->batch_desc.ptr,
                                                                         (const int2*)ctx->batch_items.ptr, n_items,
                                                                         counter, d_sc, max_nv, ctx->d_err);
        return cudaGetLastError();
    };
    goac::KTimer kt(ctx, goac::KID_MC, ctx->stream);
    if (mode == 1) {
        cudaError_t e = enqueue();
        if (e != cudaSuccess) return goac::cuda_fail(e, "k_mc_batch");
        return GOAC_OK;
    }
    if (!reuse) {
        if (ctx->batch_graph) {
            cudaGraphExecDestroy(ctx->batch_graph);
            ctx->batch_graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaStream_t cap = nullptr;
        GOAC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        const cudaStream_t saved = st;
        st = cap;   // enqueue() launches on `st`
        cudaError_t e0 = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        cudaError_t e = e0 == cudaSuccess ? enqueue() : e0;
        cudaError_t e2 = e0 == cudaSuccess ? cudaStreamEndCapture(cap, &g) : e0;
        st = saved;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return goac::cuda_fail(e, "k_mc_batch (capture)");
        }
        if (e2 != cudaSuccess) return goac::cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ctx->batch_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return goac::cuda_fail(e, "cudaGraphInstantiate");
        ctx->batch_graph_key = key;
    }
    GOAC_CUDA(cudaGraphLaunch(ctx->batch_graph, st));
    return GOAC_OK;
}

// Autotuner for the persistent batched launch: runs every chains-per-CTA
// candidate that fits in shared memory for `probe_steps` steps on scratch
// copies of the chains (the caller's configurations are not touched), times
// each with CUDA events on the context stream, and returns the fastest.
extern "C" goac_status goac_batch_mc_autotune(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs,
                                              int8_t* const* species_dev, const int32_t* chains,
                                              const double* const* kT_dev, int64_t probe_steps, int32_t precision,
                                              int32_t* best_chains_per_cta, double* best_ms)
{
    if (!ctx || !probs || n_probs <= 0 || !species_dev || !chains || !kT_dev || !best_chains_per_cta || probe_steps <= 0)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_autotune: bad argument");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    size_t sp_bytes = 0, e_count = 0;
    int max_nv = 0;
    for (int i = 0; i < n_probs; ++i) {
        if (!probs[i] || chains[i] < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_autotune: bad problem");
        sp_bytes += (((size_t)chains[i] * probs[i]->Nv) + 255) & ~(size_t)255;
        e_count += chains[i];
        max_nv = std::max(max_nv, probs[i]->Nv);
    }
    DevBuf scratch;
    goac_status rc = goac::ensure(scratch, sp_bytes + 2 * sizeof(double) * e_count + 1024);
    if (rc) return rc;
    std::vector<int8_t*> sp(n_probs);
    std::vector<double*> E(n_probs), bE(n_probs);
    {
        char* cur = (char*)scratch.ptr;
        for (int i = 0; i < n_probs; ++i) {
            sp[i] = (int8_t*)cur;
            cur += (((size_t)chains[i] * probs[i]->Nv) + 255) & ~(size_t)255;
        }
        double* d = (double*)cur;
        for (int i = 0; i < n_probs; ++i) {
            E[i] = d;
            d += chains[i];
            bE[i] = d;
            d += chains[i];
        }
    }
    const int rb = precision == GOAC_PREC_F32 ? 4 : 8;
    const size_t slot = warp_slot_bytes(max_nv, rb);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int best = -1;
    float best_t = 0.0f;
    const int cands[] = {1, 2, 4, 8, 16, 32};
    for (int cpc : cands) {
        if (slot * cpc > kSmemBudget) break;
        for (int i = 0; i < n_probs; ++i)
            if (chains[i] > 0)
                GOAC_CUDA(cudaMemcpyAsync(sp[i], species_dev[i], (size_t)chains[i] * probs[i]->Nv,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        rc = goac_batch_mc_run(ctx, probs, n_probs, sp.data(), chains, kT_dev, probe_steps, 12345u, 0, precision,
                               E.data(), bE.data(), cpc, 1);
        if (rc) break;
        cudaEventRecord(a, ctx->stream);
        rc = goac_batch_mc_run(ctx, probs, n_probs, sp.data(), chains, kT_dev, probe_steps, 12345u,
                               (uint64_t)probe_steps, precision, E.data(), bE.data(), cpc, 1);
        cudaEventRecord(b, ctx->stream);
        if (rc) break;
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (best < 0 || ms < best_t) {
            best = cpc;
            best_t = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(scratch.ptr);
    if (rc) return rc;
    if (best < 0) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_mc_autotune: no candidate fits");
    *best_chains_per_cta = best;
    if (best_ms) *best_ms = best_t;
    return GOAC_OK;
}

// Hybrid heuristic (SI, Hybrid Methods): n_cycles of replica exchange on all
// P = G R configurations followed by n_gen GA generations on them; the GA
// population (elites first) starts the next cycle's replica exchange.  Keys:
// seed + 2c for the exchange cycle c, seed + 2c + 1 for its GA (generations
// numbered from c n_gen).
extern "C" goac_status goac_hybrid_run(goac_problem* p, int8_t* species_dev, int32_t G, int32_t R,
                                       const double* kT_ladder_host, int32_t n_cycles, int32_t n_rounds,
                                       int64_t steps_per_round, int32_t n_gen, int32_t n_elite, uint32_t p_mut_u32,
                                       uint64_t seed, int32_t precision, double* E_dev)
{
    if (!p || G < 0 || R <= 0 || n_cycles < 0 || n_gen < 0 || (int64_t)G * R > GOAC_MAX_BATCH)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_hybrid_run: bad argument");
    if (G == 0) return GOAC_OK;
    if (!species_dev || !kT_ladder_host || !E_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_hybrid_run: NULL argument");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const int P = G * R;
    DevBuf perm;
    goac_status rc = goac::ensure(perm, sizeof(int32_t) * (size_t)P);
    if (rc) return rc;
    for (int c = 0; c < n_cycles && rc == GOAC_OK; ++c) {
        rc = goac_remc_run(p, species_dev, G, R, kT_ladder_host, n_rounds, steps_per_round, seed + 2 * (uint64_t)c,
                           precision, E_dev, (int32_t*)perm.ptr, nullptr);
        if (rc == GOAC_OK)
            rc = goac_ga_run(p, species_dev, E_dev, P, n_gen, n_elite, p_mut_u32, seed + 2 * (uint64_t)c + 1,
                             (uint32_t)(c * n_gen), GOAC_PREC_F64);
    }
    cudaStreamSynchronize(p->ctx->stream);
    cudaFree(perm.ptr);
    return rc;
}
