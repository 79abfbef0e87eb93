// Genetic algorithm (SI, Genetic Algorithm: roulette-wheel selection,
// crossover by random atom swaps that take half of the differences between
// the parents, random mutation, elitism), one generation per call and a
// driver that rescores every child between generations.  Every launch serves
// a list of populations (GaEntry): R independent populations of one problem
// (population r: Philox key seed + r), or one population for each of several
// problems of different sizes (the batching form).
//
// Device layout (one block or warp range per population where it says so):
//   k_ga_select   one block per population: E_min, E_max, the patience state of
//                 the population (run-level stop), F_b = floor((Emax - E_b) /
//                 (Emax - Emin) 2^24) and its running sum as exact 64-bit
//                 integers (ordered scan), so roulette selection is an exact
//                 integer search.
//   k_ga_rank     ranks by (E, index) within the population to pick the elite
//                 (O(P^2) comparisons, one warp per individual).
//   k_ga_children one warp per child (a block's warps all belong to one
//                 population): parents by binary search of the running
//                 sum, crossover in shared memory (32 sites at a time, the
//                 chunk's child values and candidate mask in registers; the
//                 draws of all remaining candidates of a chunk evaluated at
//                 once, so only taken swaps are processed one by one; the
//                 partner site j of a taken swap is the lowest position of the
//                 class with child_j == B_i and B_j != B_i, kept per species as
//                 a bitmask over class positions and found by one ballot over
//                 32 words), mutation, write-back.
//   k_ga_incr     incremental FP64 rescoring, one block per child: the
//                 potential and energy from the nearer parent's potential and
//                 the J rows of the sites where the child differs from it.
// Populations and potentials are double-buffered: generation g reads buffer
// g & 1 and writes the other, so no copy is needed between generations.
#include <algorithm>
#include <chrono>
#include <utility>
#include <vector>

#include "common.cuh"

namespace {

// Run-level stop of one population (no improvement for `patience`
// generations), kept on the device so that the generation loop needs no host
// round trip: ref = the lowest energy at the last improvement, stall = the
// generations since, stop = the population is finished (its later generations
// copy it unchanged), gens = generations run, best_gen = generation of the last
// improvement (0: the initial population), best = the current lowest energy.
struct GaTrack {
    double ref, best;
    int stall, best_gen, stop, gens;
};

// One population: its problem's data, its buffers and its place in the
// launches (child0: its first individual in the concatenation of all the
// launch's populations; block0: its first block of the children kernel).
struct GaEntry {
    const int32_t* vclass;
    const int32_t* cls_start;
    const int32_t* cls_pos;
    const int32_t* cls_rank;
    const uint32_t* wprefix;
    const double* J;          // J_vv, rows of ld doubles (incremental rescoring)
    const double* z;          // 64
    const double* phifix;     // Nv
    int8_t* pop[2];           // P x Nv each, double-buffered
    double* phi[2];           // P x Nv each (incremental rescoring), double-buffered
    double* E;                // P: energies of the current population
    unsigned long long* pre;  // P: running sum of the integer fitness
    unsigned long long* ftot; // 1
    double* mm;               // 2: E_min, E_max
    int* elite;               // n_elite
    GaTrack* track;           // 1, or null
    int32_t* parents;         // P x 2, or null
    int32_t* nswap;           // P x 2, or null
    uint64_t key;
    double E_const;
    uint32_t wtotal;
    int Nv, S, ncls, nmovable, only_movable, ld, P, n_elite, block0;
    long child0;
};

// The entry holding global index x of a prefix field (child0 or block0): the
// last entry whose start is <= x.
__device__ __forceinline__ int entry_of_child(const GaEntry* __restrict__ e, int n, long x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e[mid].child0 <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int entry_of_block(const GaEntry* __restrict__ e, int n, int x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e[mid].block0 <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One block per population: E_min / E_max, then (tracking) the patience
// update for the population as it stands after g generations, then (fitness)
// F_b = floor((Emax - E_b) / (Emax - Emin) 2^24) and its inclusive running
// sum in index order as exact 64-bit integers.
__global__ void __launch_bounds__(1024) k_ga_select(const GaEntry* __restrict__ ents, int fitness, int g,
                                                    int patience)
{
    __shared__ double smin[1024], smax[1024];
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const GaEntry& en = ents[blockIdx.x];     // one block per population
    const double* __restrict__ E = en.E;
    const int P = en.P;
    double* mm = en.mm;
    GaTrack* track = en.track;
    double lo = E[0], hi = E[0];
    for (int b = threadIdx.x; b < P; b += blockDim.x) {
        lo = fmin(lo, E[b]);
        hi = fmax(hi, E[b]);
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = blockDim.x / 2; w; w >>= 1) {
        if (threadIdx.x < w) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    const double emin = smin[0], emax = smax[0];
    if (threadIdx.x == 0) {
        mm[0] = emin;
        mm[1] = emax;
        if (track) {
            GaTrack& tr = *track;
            if (g == 0) {
                tr.ref = emin;
                tr.best = emin;
                tr.stall = tr.best_gen = tr.stop = tr.gens = 0;
            } else if (!tr.stop) {
                tr.gens = g;
                tr.best = emin;
                if (emin < tr.ref - 1e-9) {
                    tr.ref = emin;
                    tr.stall = 0;
                    tr.best_gen = g;
                } else {
                    tr.stall++;
                }
                if (patience > 0 && tr.stall >= patience) tr.stop = 1;
            }
        }
        carry = 0;
    }
    if (!fitness) return;
    __syncthreads();
    unsigned long long* pre = en.pre;
    unsigned long long* ftot = en.ftot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < P; base += blockDim.x) {
        const int b = base + threadIdx.x;
        unsigned long long f = 0;
        if (b < P) f = emax > emin ? (unsigned long long)floor((emax - E[b]) / (emax - emin) * 16777216.0) : 1ull;
        unsigned long long incl = f;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned long long v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
            unsigned long long inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            warp_tot[lane] = inc - v;   // exclusive prefix of warp totals
        }
        __syncthreads();
        const unsigned long long val = carry + warp_tot[wid] + incl;
        if (b < P) pre[b] = val;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = val;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ftot = carry;
}

// Elite selection: the rank of individual i by (E, index) is the number of j
// with E_j < E_i, or E_j == E_i and j < i; one warp per i (lanes stride over
// j, warp sum), so the O(P^2) comparisons spread over P warps.
__global__ void k_ga_rank(const GaEntry* __restrict__ ents, int n_ents, long total)
{
    const long gi = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gi >= total) return;                  // whole warps leave together
    const GaEntry& en = ents[entry_of_child(ents, n_ents, gi)];
    const int i = (int)(gi - en.child0);      // individual i of this population
    if (en.n_elite == 0) return;
    const double* E = en.E;
    const double ei = E[i];
    int rank = 0;
    for (int j = lane; j < en.P; j += 32) {
        const double ej = E[j];
        rank += (ej < ei) || (ej == ei && j < i);
    }
    rank = __reduce_add_sync(0xffffffffu, rank);
    if (lane == 0 && rank < en.n_elite) en.elite[rank] = i;
}

__device__ __forceinline__ int lower_bound_gt(const unsigned long long* pre, int P, unsigned long long t)
{
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Shared-memory slot of one child warp: child and parent B (Nv bytes each,
// 16-byte rounded) and, per species s, a bitmask over class positions p of the
// sites with child = s != B (mis[s][p / 32]).
// Block-wide copy of the class positions at the front of shared memory.
__host__ __device__ inline size_t ga_cpos_bytes(int Nv)
{
    return ((size_t)Nv * 4 + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t ga_slot_bytes(int Nv, int S)
{
    const size_t sp = ((size_t)Nv + 15) & ~(size_t)15;
    const size_t words = ((size_t)Nv + 31) / 32;
    return 2 * sp + (((size_t)S * words * 4 + 15) & ~(size_t)15);
}

// Children of generation `gen` (which reads pop[parity] of every population
// and writes pop[parity ^ 1]); the warps of a block all serve the population
// whose block range holds the block.
__global__ void k_ga_children(const GaEntry* __restrict__ ents, int n_ents, int wpb, uint32_t gen, int parity,
                              uint32_t p_mut, int* err)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const GaEntry& a = ents[entry_of_block(ents, n_ents, blockIdx.x)];
    const int Nv = a.Nv;
    // block-wide copy of the class positions (site of class position p), then one slot per warp
    int32_t* cpos = (int32_t*)smem;
    for (int q = threadIdx.x; q < Nv; q += blockDim.x) cpos[q] = a.cls_pos[q];
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = (blockIdx.x - a.block0) * wpb + wib;
    if (c >= a.P) return;
    // child c: the population's own parents, fitness sums and elite, its own Philox key
    const int8_t* popr = a.pop[parity];
    const int W = (Nv + 31) / 32;
    uint8_t* base = smem + ga_cpos_bytes(Nv) + ga_slot_bytes(Nv, a.S) * wib;
    int8_t* ch = (int8_t*)base;
    int8_t* pb = ch + (((size_t)Nv + 15) & ~(size_t)15);
    uint32_t* mis = (uint32_t*)(pb + (((size_t)Nv + 15) & ~(size_t)15));
    int8_t* out = a.pop[parity ^ 1] + (long)c * Nv;

    if (a.track && a.track->stop) {           // finished (patience): the child is the individual itself
        for (int w = lane; w < Nv; w += 32) out[w] = popr[(long)c * Nv + w];
        if (lane == 0) {
            if (a.parents) a.parents[2 * c] = a.parents[2 * c + 1] = c;
            if (a.nswap) a.nswap[2 * c] = a.nswap[2 * c + 1] = 0;
        }
        return;
    }
    if (c < a.n_elite) {
        const int src = a.elite[c];
        for (int w = lane; w < Nv; w += 32) out[w] = popr[(long)src * Nv + w];
        if (lane == 0) {
            if (a.parents) a.parents[2 * c] = a.parents[2 * c + 1] = src;
            if (a.nswap) a.nswap[2 * c] = a.nswap[2 * c + 1] = 0;
        }
        return;
    }
    const uint64_t key = a.key;
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    const uint4 x = goacd::philox(make_uint4(0u, gen, (uint32_t)c, 2u), k0, k1);
    const unsigned long long* prer = a.pre;
    const unsigned long long ftot = *a.ftot;
    const unsigned long long xa = ((unsigned long long)x.x << 32) | x.y;
    const unsigned long long xb = ((unsigned long long)x.z << 32) | x.w;
    const int A = lower_bound_gt(prer, a.P, __umul64hi(xa, ftot));
    const int B = lower_bound_gt(prer, a.P, __umul64hi(xb, ftot));
    for (int w = lane; w < Nv; w += 32) {
        ch[w] = popr[(long)A * Nv + w];
        pb[w] = popr[(long)B * Nv + w];
    }
    for (int e = lane; e < a.S * W; e += 32) mis[e] = 0u;
    __syncwarp();
    for (int q = lane; q < Nv; q += 32) {
        const int w = cpos[q];
        const int8_t s = ch[w];
        if ((unsigned)s < (unsigned)a.S && s != pb[w]) atomicOr(&mis[s * W + (q >> 5)], 1u << (q & 31));
    }
    __syncwarp();

    // Crossover: for each site i (ascending) where the child differs from B,
    // the candidate swap pairs i with the lowest class position holding B_i
    // where B differs (the lowest set bit of mis[B_i] in i's class), taken with
    // probability 1/2.  Within a chunk of 32 sites the child values and the
    // candidate mask live in registers: a taken swap changes the child at i and
    // at its partner j, and only j (if it lies later in the chunk) can change
    // its candidate bit.
    uint32_t kc = 0;
    int nsw = 0;
    // Philox cache: lane t holds block (cache_lo >> 2) + t, so the warp holds draws [cache_lo, cache_hi)
    uint4 blk = make_uint4(0, 0, 0, 0);
    uint32_t cache_lo = 0u, cache_hi = 0u;
    for (int i0 = 0; i0 < Nv; i0 += 32) {
        const int il = i0 + lane;
        // per lane: B's species, the child's species and the class position (8 + 8 + 16 bits),
        // and the class's position range (16 + 16 bits), so a candidate takes two shuffles
        uint32_t my_bcr = 0u, my_rng = 0u;
        bool bad = false;
        if (il < Nv) {
            const int k = a.vclass[il];
            const int sb = pb[il], sc = ch[il];
            bad = (unsigned)sb >= (unsigned)a.S || (unsigned)sc >= (unsigned)a.S;
            my_bcr = (uint32_t)(uint8_t)sb | ((uint32_t)(uint8_t)sc << 8) | ((uint32_t)a.cls_rank[il] << 16);
            my_rng = (uint32_t)a.cls_start[k] | ((uint32_t)a.cls_start[k + 1] << 16);
        }
        if (__any_sync(0xffffffffu, bad)) {         // not a species of the problem
            if (lane == 0) goacd::report(err, GOAC_ERR_INVALID_ARG, goac::SITE_GA, c);
            return;
        }
        uint32_t m = __ballot_sync(0xffffffffu, il < Nv && ((my_bcr ^ (my_bcr >> 8)) & 0xffu) != 0u);
        while (m) {
            // A candidate that is not taken changes nothing, and its draw is known in advance:
            // the remaining candidate of rank t (set bits of m in site order) uses draw kc + t,
            // so the warp finds the first taken one at once and only that one needs its partner.
            if (kc + 32u > cache_hi) {
                cache_lo = kc & ~3u;
                cache_hi = cache_lo + 128u;
                blk = goacd::philox(make_uint4((cache_lo >> 2) + (uint32_t)lane, gen, (uint32_t)c, 3u), k0, k1);
            }
            const uint32_t d = kc + (uint32_t)__popc(m & ((1u << lane) - 1u));
            const int src = (int)((d >> 2) - (cache_lo >> 2)) & 31;
            const uint32_t x0 = __shfl_sync(0xffffffffu, blk.x, src), x1 = __shfl_sync(0xffffffffu, blk.y, src);
            const uint32_t x2 = __shfl_sync(0xffffffffu, blk.z, src), x3 = __shfl_sync(0xffffffffu, blk.w, src);
            const uint32_t dq = d & 3u;
            const uint32_t wv = dq == 0u ? x0 : dq == 1u ? x1 : dq == 2u ? x2 : x3;
            const uint32_t tm = __ballot_sync(0xffffffffu, ((m >> lane) & 1u) != 0u && wv < 0x80000000u);
            if (tm == 0u) {                                // no further swap in this chunk
                kc += (uint32_t)__popc(m);
                break;
            }
            const int l = __ffs(tm) - 1;
            kc += (uint32_t)__popc(m & ((1u << l) - 1u)) + 1u;
            m &= l == 31 ? 0u : (~0u << (l + 1));
            const int ii = i0 + l;
            const uint32_t bcr = __shfl_sync(0xffffffffu, my_bcr, l), rng = __shfl_sync(0xffffffffu, my_rng, l);
            const int want = (int8_t)(bcr & 0xffu), old = (int8_t)((bcr >> 8) & 0xffu), pi = (int)(bcr >> 16);
            const int cs = (int)(rng & 0xffffu), ce = (int)(rng >> 16);
            const int wlo = cs >> 5, whi = (ce - 1) >> 5;
            const uint32_t* mw = mis + want * W;
            int pp = -1;
            for (int w0 = wlo; w0 <= whi; w0 += 32) {
                const int wi = w0 + lane;
                uint32_t bits = 0u;
                if (wi <= whi) {
                    bits = mw[wi];
                    if (wi == wlo) bits &= ~0u << (cs & 31);
                    if (wi == whi && (ce & 31)) bits &= (1u << (ce & 31)) - 1u;
                }
                const uint32_t mm = __ballot_sync(0xffffffffu, bits != 0u);
                if (mm) {
                    const int ll = __ffs(mm) - 1;
                    const uint32_t bw = __shfl_sync(0xffffffffu, bits, ll);
                    pp = (w0 + ll) * 32 + __ffs(bw) - 1;
                    break;
                }
            }
            if (pp < 0) {
                if (lane == 0) goacd::report(err, GOAC_ERR_INTERNAL, goac::SITE_GA, c);
                return;
            }
            const int j = cpos[pp];
            const int jl = j - i0;                      // j != ii; in this chunk iff 0 <= jl < 32
            const int pbj = pb[j];
            if (lane == l) my_bcr = (my_bcr & 0xffff00ffu) | ((uint32_t)(uint8_t)want << 8);
            if (lane == jl) my_bcr = (my_bcr & 0xffff00ffu) | ((uint32_t)(uint8_t)old << 8);
            if (jl > l && jl < 32) m = old != pbj ? (m | (1u << jl)) : (m & ~(1u << jl));
            __syncwarp();                               // every lane has read mis for this candidate
            if (lane == 0) {                            // three updates of different bits
                ch[j] = (int8_t)old;
                ch[ii] = (int8_t)want;
                atomicAnd(&mis[old * W + (pi >> 5)], ~(1u << (pi & 31)));     // i now equals B_i
                atomicAnd(&mis[want * W + (pp >> 5)], ~(1u << (pp & 31)));    // j no longer holds B_i
                if (pbj != old) atomicOr(&mis[old * W + (pp >> 5)], 1u << (pp & 31));
            }
            __syncwarp();
            ++nsw;
        }
    }
    const uint4 y = goacd::philox(make_uint4(0u, gen, (uint32_t)c, 4u), k0, k1);
    if (y.x < p_mut && a.nmovable > 0) {
        int k = a.only_movable;
        if (a.nmovable != 1) {
            const uint32_t thr = goacd::draw_below(y.y, a.wtotal);
            k = a.ncls - 1;
            for (int q = 0; q < a.ncls; ++q)
                if (a.wprefix[q] > thr) {
                    k = q;
                    break;
                }
        }
        const int start = a.cls_start[k];
        const uint32_t n = (uint32_t)(a.cls_start[k + 1] - start);
        const uint32_t pa = goacd::draw_below(y.z, n);
        const uint32_t bb = goacd::draw_below(y.w, n - 1);
        const uint32_t pbi = bb + (bb >= pa);
        const int va = cpos[start + pa], vb = cpos[start + pbi];
        __syncwarp();
        if (lane == 0) {
            const int8_t t = ch[va];
            ch[va] = ch[vb];
            ch[vb] = t;
        }
    }
    __syncwarp();
    for (int w = lane; w < Nv; w += 32) out[w] = ch[w];
    if (lane == 0) {
        if (a.parents) {
            a.parents[2 * c] = A;
            a.parents[2 * c + 1] = B;
        }
        if (a.nswap) {
            a.nswap[2 * c] = nsw;
            a.nswap[2 * c + 1] = (int32_t)kc;
        }
    }
}

// Incremental FP64 rescoring of the children (SI, Genetic Algorithm; the
// incremental form of the Eq. 2 objective): with phi = J_vv q + phi_fix kept
// for every individual, a child c and the parent P (of its two) from which it
// differs in fewer sites give
//   phi_c = phi_P + sum_{s: c_s != P_s} (z[c_s] - z[P_s]) J_vv[s][:],
//   E_c   = sum_v q_c,v (phi_c,v + phi_fix,v) + E_const,
// the changed sites taken in ascending order.  One block per child; the list
// of changed sites and charge differences sits in shared memory, each thread
// accumulates GI_R sites per pass over the list (coalesced reads of the J rows).
constexpr int GI_THREADS = 256;
constexpr int GI_R = 4;

// Children of every population: block = child (population by its child0);
// reads pop[parity] / phi[parity] (the parents) and pop[parity ^ 1] (the
// children), writes phi[parity ^ 1] and the energies.
__global__ void __launch_bounds__(GI_THREADS) k_ga_incr(const GaEntry* __restrict__ ents, int n_ents, int parity,
                                                        int* err)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const GaEntry& g = ents[entry_of_child(ents, n_ents, (long)blockIdx.x)];
    const long c = (long)blockIdx.x - g.child0;   // child c of this population
    double* dq = (double*)smem;               // Nv
    int* idx = (int*)(dq + g.Nv);             // Nv
    __shared__ int wcnt[GI_THREADS / 32][2];
    __shared__ double wsum[GI_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = GI_THREADS / 32;
    const int Nv = g.Nv;
    const int A0 = g.parents[2 * c], B0 = g.parents[2 * c + 1];
    if ((unsigned)A0 >= (unsigned)g.P || (unsigned)B0 >= (unsigned)g.P) {
        if (tid == 0) goacd::report(err, GOAC_ERR_INTERNAL, goac::SITE_GA, (int)c);
        return;
    }
    const long A = A0, B = B0;
    const int8_t* kid = g.pop[parity ^ 1] + c * Nv;
    const int8_t* pa = g.pop[parity] + A * Nv;
    const int8_t* pb = g.pop[parity] + B * Nv;
    // the nearer parent (ties: A)
    int da = 0, db = 0;
    for (int v = tid; v < Nv; v += GI_THREADS) {
        const int8_t k = kid[v];
        da += k != pa[v];
        db += k != pb[v];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        da += __shfl_xor_sync(0xffffffffu, da, o);
        db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    if (lane == 0) {
        wcnt[wid][0] = da;
        wcnt[wid][1] = db;
    }
    __syncthreads();
    int DA = 0, DB = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        DA += wcnt[w][0];
        DB += wcnt[w][1];
    }
    const bool useB = DB < DA;
    const long par = useB ? B : A;
    const int8_t* pp = useB ? pb : pa;
    __syncthreads();
    // changed sites in ascending order and their charge differences
    int M = 0;
    bool bad = false;
    for (int v0 = 0; v0 < Nv; v0 += GI_THREADS) {
        const int v = v0 + tid;
        bool f = false;
        int sk = 0, sp = 0;
        if (v < Nv) {
            sk = kid[v];
            sp = pp[v];
            f = sk != sp;
            if ((unsigned)sk >= (unsigned)g.S || (unsigned)sp >= (unsigned)g.S) {
                bad = true;
                f = false;
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wcnt[wid][0] = __popc(m);
        __syncthreads();
        int off = M, tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            off += w < wid ? wcnt[w][0] : 0;
            tot += wcnt[w][0];
        }
        if (f) {
            const int pos = off + __popc(m & ((1u << lane) - 1u));
            idx[pos] = v;
            dq[pos] = g.z[sk] - g.z[sp];
        }
        M += tot;
        __syncthreads();
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) goacd::report(err, GOAC_ERR_INVALID_ARG, goac::SITE_GA, (int)c);
        return;
    }
    double e = 0.0;
    for (int v0 = 0; v0 < Nv; v0 += GI_THREADS * GI_R) {
        double acc[GI_R];
#pragma unroll
        for (int r = 0; r < GI_R; ++r) {
            const int v = v0 + r * GI_THREADS + tid;
            acc[r] = v < Nv ? g.phi[parity][par * Nv + v] : 0.0;
        }
        for (int t = 0; t < M; ++t) {
            const double d = dq[t];
            const double* row = g.J + (long)idx[t] * g.ld;
#pragma unroll
            for (int r = 0; r < GI_R; ++r) {
                const int v = v0 + r * GI_THREADS + tid;
                if (v < Nv) acc[r] = fma(d, row[v], acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < GI_R; ++r) {
            const int v = v0 + r * GI_THREADS + tid;
            if (v < Nv) {
                g.phi[parity ^ 1][c * Nv + v] = acc[r];
                e = fma(g.z[kid[v]], acc[r] + g.phifix[v], e);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) wsum[wid] = e;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += wsum[w];
        g.E[c] = s + g.E_const;
    }
}

}  // namespace

namespace goac {

// The populations of one GA launch sequence: host and device copies of the
// entries, and the launch geometry of the children and rescoring kernels.
struct GaLaunch {
    std::vector<GaEntry> e;
    std::vector<goac_problem*> prob;   // problem of each entry
    GaEntry* dev = nullptr;
    long total = 0;                     // individuals over all entries
    int wpb = 1, blocks = 0, max_nv = 0;
    size_t smem_children = 0, smem_incr = 0;
    bool any_elite = false;
};

// Entries for R populations of P of problem p in its scratch buffer ga_buf:
// population r is rows r P .. of pop0 and E (its second buffer pop1, or rows
// of the scratch when null), Philox key seed + r.  The entries' device copy
// goes to `devbuf` (the problem's own, or a batch's).
static goac_status ga_entries(goac_problem* p, int8_t* pop0, int8_t* pop1, double* E, int R, int P, int n_elite,
                              uint64_t seed, bool incr, bool tracking, int32_t* parents, int32_t* nswap,
                              GaLaunch& L)
{
    const int Nv = p->Nv;
    const size_t RP = (size_t)R * P;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_pop = pop1 ? 0 : al(RP * Nv), b_pre = al(8 * RP), b_ftot = al(8 * (size_t)R),
                 b_mm = al(16 * (size_t)R), b_el = al(4 * (size_t)R * (n_elite > 0 ? n_elite : 1)),
                 b_tr = al(sizeof(GaTrack) * (size_t)R), b_par = (incr && !parents) ? al(8 * RP) : 0;
    goac_status rc = ensure(p->ga_buf, b_pop + b_pre + b_ftot + b_mm + b_el + b_tr + b_par + 256);
    if (rc) return rc;
    char* q = (char*)p->ga_buf.ptr;
    int8_t* pop1s = pop1 ? pop1 : (int8_t*)q;
    q += b_pop;
    unsigned long long* pre = (unsigned long long*)q;
    q += b_pre;
    unsigned long long* ftot = (unsigned long long*)q;
    q += b_ftot;
    double* mm = (double*)q;
    q += b_mm;
    int* elite = (int*)q;
    q += b_el;
    GaTrack* track = (GaTrack*)q;
    q += b_tr;
    int32_t* par = parents ? parents : (incr ? (int32_t*)q : nullptr);
    double* phi0 = nullptr;
    if (incr) {
        rc = ensure(p->ga_incr, 2 * sizeof(double) * RP * Nv + 256);
        if (rc) return rc;
        phi0 = (double*)p->ga_incr.ptr;
    }
    for (int r = 0; r < R; ++r) {
        GaEntry e{};
        e.vclass = p->vclass_dev;
        e.cls_start = p->cls_start_dev;
        e.cls_pos = p->cls_pos_dev;
        e.cls_rank = p->cls_rank_dev;
        e.wprefix = p->wprefix_dev;
        e.J = p->J_vv;
        e.z = p->z_dev;
        e.phifix = p->phifix;
        e.pop[0] = pop0 + (size_t)r * P * Nv;
        e.pop[1] = pop1s + (size_t)r * P * Nv;
        e.phi[0] = incr ? phi0 + (size_t)r * P * Nv : nullptr;
        e.phi[1] = incr ? phi0 + RP * Nv + (size_t)r * P * Nv : nullptr;
        e.E = E + (size_t)r * P;
        e.pre = pre + (size_t)r * P;
        e.ftot = ftot + r;
        e.mm = mm + 2 * r;
        e.elite = elite + (size_t)r * (n_elite > 0 ? n_elite : 1);
        e.track = tracking ? track + r : nullptr;
        e.parents = par ? par + 2 * (size_t)r * P : nullptr;
        e.nswap = nswap ? nswap + 2 * (size_t)r * P : nullptr;
        e.key = seed + (uint64_t)r;
        e.E_const = p->E_const;
        e.wtotal = p->wtotal;
        e.Nv = Nv;
        e.S = p->S;
        e.ncls = p->ncls;
        e.nmovable = p->nmovable;
        e.only_movable = p->only_movable;
        e.ld = p->Nv_pad;
        e.P = P;
        e.n_elite = n_elite;
        L.e.push_back(e);
        L.prob.push_back(p);
    }
    return GOAC_OK;
}

// Launch geometry of the entries and their device copy in `devbuf`: warps
// (children) per block a power of two up to 8, small enough that the grid
// spreads over at least two blocks per SM, within 96 KB of shared memory for
// the largest population's working set.
static goac_status ga_finalize(goac_ctx* ctx, GaLaunch& L, DevBuf& devbuf)
{
    size_t slot = 0, cpos = 0;
    L.total = 0;
    L.max_nv = 0;
    L.any_elite = false;
    for (const GaEntry& e : L.e) {
        slot = std::max(slot, ga_slot_bytes(e.Nv, e.S));
        cpos = std::max(cpos, ga_cpos_bytes(e.Nv));
        L.total += e.P;
        L.max_nv = std::max(L.max_nv, e.Nv);
        L.any_elite = L.any_elite || e.n_elite > 0;
    }
    // (this bounds Nv to at most 33,432, so class positions fit the 16-bit fields the kernel packs)
    if (slot + cpos > 200 * 1024 || L.max_nv > 65535)
        return fail(GOAC_ERR_INVALID_ARG, "goac_ga_generation: Nv too large");
    int wpb = 8;
    while (wpb > 1 && (cpos + (size_t)wpb * slot > 96 * 1024 || (L.total + wpb - 1) / wpb < 2 * ctx->num_sms)) wpb >>= 1;
    L.wpb = wpb;
    L.smem_children = cpos + slot * wpb;
    L.smem_incr = (sizeof(double) + sizeof(int)) * (size_t)L.max_nv;
    long child0 = 0;
    int block0 = 0;
    for (GaEntry& e : L.e) {
        e.child0 = child0;
        e.block0 = block0;
        child0 += e.P;
        block0 += (e.P + wpb - 1) / wpb;
    }
    L.blocks = block0;
    goac_status rc = ensure(devbuf, sizeof(GaEntry) * L.e.size() + 64);
    if (rc) return rc;
    L.dev = (GaEntry*)devbuf.ptr;
    GOAC_CUDA(cudaMemcpyAsync(L.dev, L.e.data(), sizeof(GaEntry) * L.e.size(), cudaMemcpyHostToDevice, ctx->stream));
    return GOAC_OK;
}

// One generation of every entry: generation number gen reads buffers
// `parity` and writes the other; g / patience drive the run-level stop.
static goac_status ga_gen_launch(goac_ctx* ctx, const GaLaunch& L, uint32_t gen, int parity, uint32_t p_mut, int g,
                                 int patience)
{
    cudaStream_t st = ctx->stream;
    const int n = (int)L.e.size();
    goac::launch(k_ga_select, n, 1024, 0, st, (const GaEntry*)L.dev, 1, g, patience);
    if (L.any_elite) goac::launch(k_ga_rank, (int)((L.total + 7) / 8), 256, 0, st, (const GaEntry*)L.dev, n, L.total);
    GOAC_LAUNCH_CHECK("ga prep");
    GOAC_CUDA(cudaFuncSetAttribute(k_ga_children, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    KTimer kt(ctx, KID_GA, st);
    goac::launch(k_ga_children, L.blocks, 32 * L.wpb, L.smem_children, st, (const GaEntry*)L.dev, n, L.wpb, gen,
                 parity, p_mut, ctx->d_err);
    GOAC_LAUNCH_CHECK("k_ga_children");
    return GOAC_OK;
}

struct GaRunOpts {
    int n_gen, n_elite, precision, patience;
    uint32_t p_mut, gen0;
    double time_budget_s;
};

// GA run over the entries of L (populations of one problem, or of several
// problems when every entry's rescoring is incremental): initial scoring,
// then per generation the children and their rescoring, dense (goac_score in
// the requested form over the single problem's populations) or incremental in
// FP64 (k_ga_incr from the nearer parent's potential; the potentials of the
// starting populations by the FP64 scoring GEMM).  With tracking, the select
// kernel keeps each population's patience state on the device and finished
// populations are copied unchanged; the host looks at the states every 8
// generations (one small copy) to stop launching once every population has
// finished or the wall-clock budget is spent.  The final population ends up in
// each entry's pop[0].
static goac_status ga_run_core(goac_ctx* ctx, GaLaunch& L, const GaRunOpts& o, goac_ga_stats* stats)
{
    cudaStream_t st = ctx->stream;
    const bool incr = o.precision == GOAC_PREC_F64_INCR;
    const bool tracking = L.e[0].track != nullptr;
    const int n = (int)L.e.size();
    if (incr && L.smem_incr > 200 * 1024)
        return fail(GOAC_ERR_UNSUPPORTED, "goac_ga_run: incremental rescoring needs Nv <= 17066");
    goac_status rc = GOAC_OK;
    // starting energies (and potentials), per run of entries that share a problem
    for (int i = 0; i < n && !rc;) {
        int j = i;
        while (j < n && L.prob[j] == L.prob[i] && L.e[j].pop[0] == L.e[i].pop[0] + (size_t)(j - i) * L.e[i].P * L.e[i].Nv)
            ++j;
        const int RP = L.e[i].P * (j - i);
        rc = incr ? score_f64(L.prob[i], L.e[i].pop[0], RP, L.e[i].E, L.e[i].phi[0])
                  : goac_score(L.prob[i], L.e[i].pop[0], RP, o.precision, L.e[i].E);
        i = j;
    }
    if (rc) return rc;
    if (incr) GOAC_CUDA(cudaFuncSetAttribute(k_ga_incr, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    const auto t_start = std::chrono::steady_clock::now();
    std::vector<GaTrack> host(tracking ? n : 0);
    int stop_reason = 0, g = 0;
    for (; g < o.n_gen; ++g) {
        const int parity = g & 1;
        rc = ga_gen_launch(ctx, L, o.gen0 + (uint32_t)g, parity, o.p_mut, g, o.patience);
        if (rc) return rc;
        if (incr) {
            {
                KTimer kt(ctx, KID_GA_INCR, st);
                goac::launch(k_ga_incr, (int)L.total, GI_THREADS, L.smem_incr, st, (const GaEntry*)L.dev, n, parity,
                             ctx->d_err);
            }
            GOAC_LAUNCH_CHECK("k_ga_incr");
        } else {
            // a single problem: its populations' second buffers are contiguous
            rc = goac_score(L.prob[0], L.e[0].pop[parity ^ 1], (int)L.total, o.precision, L.e[0].E);
            if (rc) return rc;
        }
        if (tracking && (o.patience > 0 || o.time_budget_s > 0.0) && (g + 1) % 8 == 0 && g + 1 < o.n_gen) {
            for (int r = 0; r < n; ++r)
                GOAC_CUDA(cudaMemcpyAsync(&host[r], L.e[r].track, sizeof(GaTrack), cudaMemcpyDeviceToHost, st));
            GOAC_CUDA(cudaStreamSynchronize(st));
            bool all = o.patience > 0;
            for (int r = 0; r < n && all; ++r) all = host[r].stop != 0;
            if (all) {
                ++g;
                break;
            }
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (o.time_budget_s > 0.0 && el >= o.time_budget_s) {
                stop_reason = 2;
                ++g;
                break;
            }
        }
    }
    // the final populations into pop[0]
    if (g & 1)
        for (int i = 0; i < n;) {
            int j = i;
            while (j < n && L.prob[j] == L.prob[i] &&
                   L.e[j].pop[1] == L.e[i].pop[1] + (size_t)(j - i) * L.e[i].P * L.e[i].Nv &&
                   L.e[j].pop[0] == L.e[i].pop[0] + (size_t)(j - i) * L.e[i].P * L.e[i].Nv)
                ++j;
            GOAC_CUDA(cudaMemcpyAsync(L.e[i].pop[0], L.e[i].pop[1], (size_t)(j - i) * L.e[i].P * L.e[i].Nv,
                                      cudaMemcpyDeviceToDevice, st));
            i = j;
        }
    if (!tracking) return GOAC_OK;
    // the state after the last generation run
    goac::launch(k_ga_select, n, 1024, 0, st, (const GaEntry*)L.dev, 0, g, o.patience);
    GOAC_LAUNCH_CHECK("k_ga_select (final)");
    if (stats) {
        for (int r = 0; r < n; ++r)
            GOAC_CUDA(cudaMemcpyAsync(&host[r], L.e[r].track, sizeof(GaTrack), cudaMemcpyDeviceToHost, st));
        GOAC_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < n; ++r) {
            stats[r].generations = host[r].stop ? host[r].gens : g;
            stats[r].best_generation = host[r].best_gen;
            stats[r].stop_reason = host[r].stop ? 1 : stop_reason;
            stats[r].reserved = 0;
            stats[r].best_E = host[r].best;
        }
    }
    return GOAC_OK;
}

}  // namespace goac

extern "C" goac_status goac_ga_generation(goac_problem* p, const int8_t* pop_dev, const double* E_dev, int32_t P,
                                          int32_t n_elite, uint32_t p_mut_u32, uint32_t gen, uint64_t seed,
                                          int8_t* children_dev, int32_t* parents_dev, int32_t* nswap_dev)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_generation: NULL problem");
    if (P < 0 || P > GOAC_MAX_BATCH || n_elite < 0 || n_elite > P) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_generation: bad sizes");
    if (P == 0) return GOAC_OK;
    if (!pop_dev || !E_dev || !children_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_generation: NULL");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    goac::GaLaunch L;
    goac_status rc = goac::ga_entries(p, const_cast<int8_t*>(pop_dev), children_dev, const_cast<double*>(E_dev), 1, P,
                                      n_elite, seed, false, false, parents_dev, nswap_dev, L);
    if (!rc) rc = goac::ga_finalize(p->ctx, L, p->ga_dev);
    if (!rc) rc = goac::ga_gen_launch(p->ctx, L, gen, 0, p_mut_u32, 0, 0);
    return rc;
}

static goac_status ga_run_problem(goac_problem* p, int8_t* pop_dev, double* E_dev, int32_t R, int32_t P,
                                  const goac::GaRunOpts& o, uint64_t seed, goac_ga_stats* stats)
{
    if (!p) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run: NULL problem");
    if (R < 0 || P < 0 || (int64_t)R * P > GOAC_MAX_BATCH || o.n_gen < 0 || o.n_elite < 0 || o.n_elite > P ||
        o.patience < 0 || !(o.time_budget_s >= 0.0))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run: bad sizes or parameters");
    if (R == 0 || P == 0) return GOAC_OK;
    if (!pop_dev || !E_dev) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run: NULL");
    GOAC_CUDA(cudaSetDevice(p->ctx->device));
    const bool incr = o.precision == GOAC_PREC_F64_INCR;
    const bool tracking = o.patience > 0 || o.time_budget_s > 0.0 || stats != nullptr;
    goac::GaLaunch L;
    goac_status rc = goac::ga_entries(p, pop_dev, nullptr, E_dev, R, P, o.n_elite, seed, incr, tracking, nullptr,
                                      nullptr, L);
    if (!rc) rc = goac::ga_finalize(p->ctx, L, p->ga_dev);
    if (!rc) rc = goac::ga_run_core(p->ctx, L, o, stats);
    return rc;
}

extern "C" goac_status goac_ga_run_populations(goac_problem* p, int8_t* pop_dev, double* E_dev, int32_t R,
                                               int32_t P, int32_t n_gen, int32_t n_elite, uint32_t p_mut_u32,
                                               uint64_t seed, uint32_t gen0, int32_t precision)
{
    goac::GaRunOpts o{n_gen, n_elite, precision, 0, p_mut_u32, gen0, 0.0};
    return ga_run_problem(p, pop_dev, E_dev, R, P, o, seed, nullptr);
}

extern "C" goac_status goac_ga_run(goac_problem* p, int8_t* pop_dev, double* E_dev, int32_t P, int32_t n_gen,
                                   int32_t n_elite, uint32_t p_mut_u32, uint64_t seed, uint32_t gen0,
                                   int32_t precision)
{
    return goac_ga_run_populations(p, pop_dev, E_dev, 1, P, n_gen, n_elite, p_mut_u32, seed, gen0, precision);
}

extern "C" goac_status goac_ga_run_ex(goac_problem* p, int8_t* pop_dev, double* E_dev, int32_t R,
                                      const goac_ga_params* prm, uint64_t seed, int32_t topk, int32_t* top_idx_dev,
                                      double* topE_dev, goac_ga_stats* stats_host)
{
    if (!p || !prm) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run_ex: NULL problem or parameters");
    const int32_t P = prm->P;
    if (topk < 0 || (R > 0 && P > 0 && topk > std::min(P, 1024)))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run_ex: topk must be in 0 .. min(P, 1024)");
    if (R > 0 && P > 0 && topk > 0 && (!top_idx_dev || !topE_dev))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_ga_run_ex: NULL");
    goac::GaRunOpts o{prm->n_gen, prm->n_elite, prm->precision, prm->patience, prm->p_mut_u32, prm->gen0,
                      prm->time_budget_s};
    goac_status rc = ga_run_problem(p, pop_dev, E_dev, R, P, o, seed, stats_host);
    if (rc || topk == 0 || R == 0 || P == 0) return rc;
    for (int r = 0; r < R && !rc; ++r)
        rc = goac_topk_rescore(p, pop_dev + (size_t)r * P * p->Nv, P, E_dev + (size_t)r * P, topk,
                               top_idx_dev + (size_t)r * topk, topE_dev + (size_t)r * topk);
    return rc;
}

extern "C" goac_status goac_batch_ga_run(goac_ctx* ctx, goac_problem* const* probs, int32_t n_probs,
                                         int8_t* const* pop_dev, double* const* E_dev, const int32_t* P,
                                         int32_t n_gen, int32_t n_elite, uint32_t p_mut_u32, uint64_t seed,
                                         uint32_t gen0, int32_t precision)
{
    if (!ctx || n_probs < 0 || (n_probs > 0 && (!probs || !pop_dev || !E_dev || !P)) || n_gen < 0 || n_elite < 0)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_ga_run: bad argument");
    if (precision != GOAC_PREC_F64_INCR)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_ga_run: precision must be GOAC_PREC_F64_INCR");
    int64_t total = 0;
    for (int i = 0; i < n_probs; ++i) {
        if (!probs[i] || probs[i]->ctx != ctx || P[i] < 0 || n_elite > P[i])
            return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_ga_run: bad problem or population size");
        if (P[i] > 0 && (!pop_dev[i] || !E_dev[i])) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_ga_run: NULL");
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i] && P[i] > 0 && P[j] > 0)
                return goac::fail(GOAC_ERR_INVALID_ARG,
                                  "goac_batch_ga_run: a problem appears twice (use goac_ga_run_populations)");
        total += P[i];
    }
    if (total > GOAC_MAX_BATCH) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_batch_ga_run: too many individuals");
    if (total == 0) return GOAC_OK;
    GOAC_CUDA(cudaSetDevice(ctx->device));
    goac::GaLaunch L;
    goac_status rc = GOAC_OK;
    for (int i = 0; i < n_probs && !rc; ++i)
        if (P[i] > 0)
            rc = goac::ga_entries(probs[i], pop_dev[i], nullptr, E_dev[i], 1, P[i], n_elite, seed + (uint64_t)i, true,
                                  false, nullptr, nullptr, L);
    if (!rc) rc = goac::ga_finalize(ctx, L, ctx->ga_dev);
    goac::GaRunOpts o{n_gen, n_elite, precision, 0, p_mut_u32, gen0, 0.0};
    if (!rc) rc = goac::ga_run_core(ctx, L, o, nullptr);
    return rc;
}
