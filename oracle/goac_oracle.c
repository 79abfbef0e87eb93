/*
 * goac_oracle.c -- plain, slow, obviously-correct CPU FP64 oracle for the
 * pairwise (second-order) Coulomb cluster-expansion optimiser of
 * "Optimization of Coulomb Energies in Gigantic Configurational Spaces of
 * Multi-Element Ionic Crystals" (GOAC).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; the two
 * only meet through the seeded input generators (goac_synth.py), which hold
 * none of the method's arithmetic.
 *
 * Compiled with -ffp-contract=off so that x86-64 and aarch64 hosts give the
 * same bits (no silent fused multiply-adds).
 *
 * Pins (tests/test_oracle_*.py) and parity status of each function:
 *   orc_philox4x32_10      pinned: published known-answer vectors (SC'11).
 *   orc_cell_geometry      pinned: a_i . b_j = 2 pi delta_ij, volume of cubes.
 *   orc_ewald_J[_entries]  pinned: Madelung constants of rocksalt, CsCl and
 *                          zincblende; alpha-independence; symmetry;
 *                          translation invariance; direct Ewald energy.
 *   orc_ewald_energy       pinned: same Madelung constants (independent of J).
 *   orc_score, orc_qJq     pinned: equals orc_ewald_energy of the configuration.
 *   orc_fixed_split        pinned: split form equals full q^T J q.
 *   orc_ce_from_J,
 *   orc_ce_from_substructures, orc_ce_energy
 *                          pinned: Eq. 2 energy equals direct Ewald energy;
 *                          sub-structure coefficients equal J-based ones.
 *   orc_delta_E            pinned: equals E(after) - E(before).
 *   orc_hybrid_run         pinned: composition of orc_remc_run and orc_ga_run
 *                          (checked against calling them in turn); finds the
 *                          brute-forced minimum.
 *   orc_gd_run             pinned: result is a local minimum by brute force over
 *                          all swaps; energies non-increasing; ground state is
 *                          a fixed point.
 *   orc_sa_run             pinned: constant schedule equals orc_mc_run; kT -> 0
 *                          end is a descent; schedule endpoints.
 *   orc_remc_run           pinned: detailed balance of the exchange (two-level
 *                          chi^2), perm stays a permutation, R = 1 equals MC.
 *   orc_mc_run             pinned: Boltzmann visit frequencies (chi^2) on a
 *                          brute-forced cell; count preservation; E tracking;
 *                          the same trajectories as orc_mc_run_literal (the
 *                          paper's rule without the tie band and log form).
 *   orc_mc_run_literal,
 *   orc_gd_run_literal     the literal-rule twins: checked against their own
 *                          definitions by the same properties (Boltzmann
 *                          visits, local minima by fresh rescoring).
 *   orc_mc_run_ex,
 *   orc_ga_run_ex          patience and statistics: equal orc_mc_run /
 *                          orc_ga_run when patience is 0 or never reached;
 *                          the stop step / generation is checked against the
 *                          rule recomputed from the recorded energy traces.
 *   orc_ga_generation      pinned: count preservation, elitism, inheritance
 *                          of common sites, 50 % swap acceptance (statistical).
 *   orc_random_configs     pinned: counts; uniformity (chi^2) on small cells.
 *   orc_energy_grad        pinned: central finite differences; dE/dq = 2 J q.
 *   orc_round_to_counts    pinned: counts; brute-force optimality of the
 *                          greedy on a one-hot input.
 *   orc_enumerate          pinned: exact count of Eq. 1; closed-form NaCl.
 *   orc_enumerate_two_species  pinned: equals orc_enumerate (minimum, its
 *                          minimisers, the count) on cells small enough for both.
 *   orc_log10_configurations  pinned: Table 1 and the NaCl / FeSbO4 counts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
/* Energy changes within this many eV of zero count as zero (Metropolis rule). */
#define ORC_DE_ZERO 1e-9

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Counter-based: out = f(counter, key).        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {           /* key schedule: Weyl sequence */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t x[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, x);
}

/* Uniform integer in [0, n) from a 32-bit draw by the multiply-high map. */
static uint32_t draw_below(uint32_t x, uint32_t n)
{
    return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Geometry of the periodic supercell.  A is row-major 3x3 whose rows are   */
/* the lattice vectors a1, a2, a3 (Angstrom).  B rows are the reciprocal     */
/* vectors b_i = 2 pi (a_j x a_k) / V, so that a_i . b_j = 2 pi delta_ij.   */
/* ------------------------------------------------------------------------ */
static void cross3(const double* u, const double* v, double* w)
{
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

void orc_cell_geometry(const double A[9], double B[9], double* V)
{
    double c23[3], c31[3], c12[3];
    cross3(A + 3, A + 6, c23);
    cross3(A + 6, A + 0, c31);
    cross3(A + 0, A + 3, c12);
    double vol = A[0] * c23[0] + A[1] * c23[1] + A[2] * c23[2];
    for (int d = 0; d < 3; ++d) {
        B[0 + d] = 2.0 * ORC_PI * c23[d] / vol;
        B[3 + d] = 2.0 * ORC_PI * c31[d] / vol;
        B[6 + d] = 2.0 * ORC_PI * c12[d] / vol;
    }
    *V = fabs(vol);
}

void orc_frac_to_cart(const double A[9], const double* frac, int64_t n, double* cart)
{
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c)
            cart[3 * i + c] = frac[3 * i + 0] * A[0 + c] + frac[3 * i + 1] * A[3 + c] + frac[3 * i + 2] * A[6 + c];
}

/* Minimum-image fractional difference f_j - f_i, each component in [-1/2, 1/2). */
static void frac_diff(const double* fi, const double* fj, double* d)
{
    for (int c = 0; c < 3; ++c) {
        double x = fj[c] - fi[c];
        d[c] = x - floor(x + 0.5);
    }
}

/* ------------------------------------------------------------------------ */
/* Reciprocal lattice vectors k = m1 b1 + m2 b2 + m3 b3, k != 0, |k| <= kcut */
/* (all of them, both k and -k; a vector on the sphere |k| = kcut counts).  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double* k;   /* n x 3 */
} kset;

static int kvec_in_sphere(double k2, double kcut)
{
    return k2 <= kcut * kcut * (1.0 + 1e-12);
}

static kset make_kset(const double A[9], double kcut)
{
    double B[9], V;
    orc_cell_geometry(A, B, &V);
    int mmax[3];
    for (int d = 0; d < 3; ++d) {
        double alen = sqrt(A[3 * d] * A[3 * d] + A[3 * d + 1] * A[3 * d + 1] + A[3 * d + 2] * A[3 * d + 2]);
        mmax[d] = (int)floor(kcut * alen / (2.0 * ORC_PI)) + 1;
    }
    int cap = (2 * mmax[0] + 1) * (2 * mmax[1] + 1) * (2 * mmax[2] + 1);
    kset ks;
    ks.n = 0;
    ks.k = (double*)malloc(sizeof(double) * 3 * (size_t)(cap > 0 ? cap : 1));
    for (int m1 = -mmax[0]; m1 <= mmax[0]; ++m1)
        for (int m2 = -mmax[1]; m2 <= mmax[1]; ++m2)
            for (int m3 = -mmax[2]; m3 <= mmax[2]; ++m3) {
                if (m1 == 0 && m2 == 0 && m3 == 0) continue;
                double k[3];
                for (int c = 0; c < 3; ++c) k[c] = m1 * B[c] + m2 * B[3 + c] + m3 * B[6 + c];
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (!kvec_in_sphere(k2, kcut)) continue;
                ks.k[3 * ks.n + 0] = k[0];
                ks.k[3 * ks.n + 1] = k[1];
                ks.k[3 * ks.n + 2] = k[2];
                ks.n++;
            }
    return ks;
}

int orc_count_kvectors(const double A[9], double kcut)
{
    kset ks = make_kset(A, kcut);
    int n = ks.n;
    free(ks.k);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Ewald pair matrix J (Section "Cluster Expansion of Coulomb Energy": the  */
/* second-order expansion is exact for point charges and its coefficients  */
/* are Ewald energies).  With q the charges of all N sites, the periodic    */
/* Coulomb energy with a neutralising background is E = q^T J q, where      */
/*                                                                          */
/*  J_ij = ke/2 * [ sum'_n erfc(alpha |d+n|) / |d+n|                        */
/*                + (4 pi / V) sum_{k != 0, |k|<=kcut} exp(-k^2/4alpha^2)    */
/*                                              / k^2 * cos(k . d)          */
/*                - (2 alpha / sqrt(pi)) delta_ij                           */
/*                - pi / (V alpha^2) ]                                      */
/*                                                                          */
/* d = minimum-image r_j - r_i, n runs over the lattice translations with   */
/* |n_a| <= nimg[a], and the prime drops n = 0 when i == j.                 */
/* ------------------------------------------------------------------------ */
static double J_entry(const double A[9], double V, const double* frac, int64_t i, int64_t j,
                      double alpha, const int nimg[3], const kset* ks, double ke)
{
    double df[3], d[3];
    frac_diff(frac + 3 * i, frac + 3 * j, df);
    for (int c = 0; c < 3; ++c) d[c] = df[0] * A[0 + c] + df[1] * A[3 + c] + df[2] * A[6 + c];

    double real = 0.0;
    for (int n1 = -nimg[0]; n1 <= nimg[0]; ++n1)
        for (int n2 = -nimg[1]; n2 <= nimg[1]; ++n2)
            for (int n3 = -nimg[2]; n3 <= nimg[2]; ++n3) {
                if (i == j && n1 == 0 && n2 == 0 && n3 == 0) continue;
                double r[3];
                for (int c = 0; c < 3; ++c) r[c] = d[c] + n1 * A[0 + c] + n2 * A[3 + c] + n3 * A[6 + c];
                double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                real += erfc(alpha * rr) / rr;
            }

    double recip = 0.0;
    for (int t = 0; t < ks->n; ++t) {
        const double* k = ks->k + 3 * t;
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        recip += exp(-k2 / (4.0 * alpha * alpha)) / k2 * cos(k[0] * d[0] + k[1] * d[1] + k[2] * d[2]);
    }
    recip *= 4.0 * ORC_PI / V;

    double self = (i == j) ? -2.0 * alpha / sqrt(ORC_PI) : 0.0;
    double bg = -ORC_PI / (V * alpha * alpha);
    return 0.5 * ke * (real + recip + self + bg);
}

/* Selected entries J[pairs[2t], pairs[2t+1]] (for sampled parity at full size). */
int orc_ewald_J_entries(const double A[9], const double* frac, int64_t N, double alpha, const int nimg[3],
                        double kcut, double ke, const int64_t* pairs, int64_t npairs, double* out)
{
    double B[9], V;
    orc_cell_geometry(A, B, &V);
    kset ks = make_kset(A, kcut);
    for (int64_t t = 0; t < npairs; ++t) {
        int64_t i = pairs[2 * t], j = pairs[2 * t + 1];
        if (i < 0 || j < 0 || i >= N || j >= N) { free(ks.k); return -1; }
        out[t] = J_entry(A, V, frac, i, j, alpha, nimg, &ks, ke);
    }
    free(ks.k);
    return 0;
}

/* Full N x N row-major J, every entry by the definition above. */
int orc_ewald_J(const double A[9], const double* frac, int64_t N, double alpha, const int nimg[3],
                double kcut, double ke, double* J)
{
    double B[9], V;
    orc_cell_geometry(A, B, &V);
    kset ks = make_kset(A, kcut);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j)
            J[i * N + j] = J_entry(A, V, frac, i, j, alpha, nimg, &ks, ke);
    free(ks.k);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Direct Ewald energy of one set of charges, computed without J:          */
/*   E = ke/2 sum_ij sum'_n q_i q_j erfc(alpha r)/r                         */
/*     + ke (2 pi / V) sum_{k != 0} exp(-k^2/4alpha^2)/k^2 |S(k)|^2,        */
/*       S(k) = sum_j q_j exp(i k . r_j)   (structure factor)               */
/*     - ke alpha/sqrt(pi) sum_i q_i^2 - ke pi Q^2 / (2 V alpha^2).        */
/* ------------------------------------------------------------------------ */
double orc_ewald_energy(const double A[9], const double* frac, const double* q, int64_t N, double alpha,
                        const int nimg[3], double kcut, double ke)
{
    double B[9], V;
    orc_cell_geometry(A, B, &V);
    kset ks = make_kset(A, kcut);

    double real = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            if (q[i] == 0.0 || q[j] == 0.0) continue;
            double df[3], d[3];
            frac_diff(frac + 3 * i, frac + 3 * j, df);
            for (int c = 0; c < 3; ++c) d[c] = df[0] * A[0 + c] + df[1] * A[3 + c] + df[2] * A[6 + c];
            double s = 0.0;
            for (int n1 = -nimg[0]; n1 <= nimg[0]; ++n1)
                for (int n2 = -nimg[1]; n2 <= nimg[1]; ++n2)
                    for (int n3 = -nimg[2]; n3 <= nimg[2]; ++n3) {
                        if (i == j && n1 == 0 && n2 == 0 && n3 == 0) continue;
                        double r[3];
                        for (int c = 0; c < 3; ++c) r[c] = d[c] + n1 * A[0 + c] + n2 * A[3 + c] + n3 * A[6 + c];
                        double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                        s += erfc(alpha * rr) / rr;
                    }
            real += q[i] * q[j] * s;
        }
    real *= 0.5 * ke;

    double *cart = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    orc_frac_to_cart(A, frac, N, cart);
    double recip = 0.0;
    for (int t = 0; t < ks.n; ++t) {
        const double* k = ks.k + 3 * t;
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double sre = 0.0, sim = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double ph = k[0] * cart[3 * j] + k[1] * cart[3 * j + 1] + k[2] * cart[3 * j + 2];
            sre += q[j] * cos(ph);
            sim += q[j] * sin(ph);
        }
        recip += exp(-k2 / (4.0 * alpha * alpha)) / k2 * (sre * sre + sim * sim);
    }
    recip *= ke * 2.0 * ORC_PI / V;
    free(cart);
    free(ks.k);

    double q2 = 0.0, Q = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        q2 += q[i] * q[i];
        Q += q[i];
    }
    double self = -ke * alpha / sqrt(ORC_PI) * q2;
    double bg = -ke * ORC_PI * Q * Q / (2.0 * V * alpha * alpha);
    return real + recip + self + bg;
}

/* ------------------------------------------------------------------------ */
/* Quadratic form and configurations.                                      */
/* A problem: N sites; site_class[i] = -1 for a fixed ion of charge        */
/* fixed_q[i], else the index of the (partially occupied) site class.      */
/* S species with charges z[s].  A configuration assigns one species index  */
/* to every variable site, variable sites taken in ascending site order.    */
/* ------------------------------------------------------------------------ */
double orc_qJq(const double* J, const double* q, int64_t N)
{
    double e = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double row = 0.0;
        for (int64_t j = 0; j < N; ++j) row += J[i * N + j] * q[j];
        e += q[i] * row;
    }
    return e;
}

static int64_t count_variable(const int32_t* site_class, int64_t N)
{
    int64_t nv = 0;
    for (int64_t i = 0; i < N; ++i) nv += site_class[i] >= 0;
    return nv;
}

void orc_config_charges(int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                        const int8_t* species_v, double* q)
{
    int64_t v = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (site_class[i] < 0) q[i] = fixed_q[i];
        else q[i] = z[(int)species_v[v++]];
    }
}

/* Energies of B configurations (species: B x Nv, config-major), E = q^T J q. */
void orc_score(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
               const int8_t* species, int64_t B, double* E)
{
    int64_t nv = count_variable(site_class, N);
    double* q = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t b = 0; b < B; ++b) {
        orc_config_charges(N, site_class, fixed_q, z, species + b * nv, q);
        E[b] = orc_qJq(J, q, N);
    }
    free(q);
}

/* Fixed-site part of the expansion (the paper's zero-order term and the    */
/* fixed-ion share of the first-order term): phi_fix[v] = sum_f J[v,f] q_f, */
/* E_const = q_f^T J_ff q_f.  Then E = q_v^T J_vv q_v + 2 q_v.phi_fix + E_const. */
void orc_fixed_split(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q,
                     double* phi_fix, double* E_const)
{
    int64_t v = 0;
    double ec = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t f = 0; f < N; ++f)
            if (site_class[f] < 0) s += J[i * N + f] * fixed_q[f];
        if (site_class[i] >= 0) phi_fix[v++] = s;
        else ec += fixed_q[i] * s;
    }
    *E_const = ec;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: E_tot = E_const + sum alpha_{s,j} x_{s,j}                         */
/*               + sum_{(s,j) < (t,l)} beta_{s,j,t,l} x_{s,j} x_{t,l}       */
/* over binary x with one entry per (species, variable position).          */
/* Coefficients stored densely: alpha[v*S + s], beta[(v*S+s)*(Nv*S) + w*S+t] */
/* (only pairs of distinct positions v < w are used).                       */
/* ------------------------------------------------------------------------ */

/* Coefficients read off J. */
void orc_ce_from_J(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                   int32_t S, double* E_const, double* alpha, double* beta)
{
    int64_t nv = count_variable(site_class, N);
    int64_t* vidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    double* phi_fix = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    int64_t v = 0;
    for (int64_t i = 0; i < N; ++i)
        if (site_class[i] >= 0) vidx[v++] = i;
    orc_fixed_split(J, N, site_class, fixed_q, phi_fix, E_const);
    int64_t M = nv * S;
    for (int64_t a = 0; a < nv; ++a)
        for (int s = 0; s < S; ++s) {
            int64_t i = vidx[a];
            alpha[a * S + s] = z[s] * z[s] * J[i * N + i] + 2.0 * z[s] * phi_fix[a];
        }
    for (int64_t r = 0; r < M * M; ++r) beta[r] = 0.0;
    for (int64_t a = 0; a < nv; ++a)
        for (int64_t b = a + 1; b < nv; ++b)
            for (int s = 0; s < S; ++s)
                for (int t = 0; t < S; ++t)
                    beta[(a * S + s) * M + b * S + t] = 2.0 * z[s] * z[t] * J[vidx[a] * N + vidx[b]];
    free(vidx);
    free(phi_fix);
}

/* Coefficients as the paper builds them: Ewald energies of sub-structures  */
/* (fixed ions only; plus one placed ion; plus two placed ions), with the   */
/* lower-order energies subtracted to avoid double counting.  Sub-structures */
/* are not neutral; the neutralising background makes each energy defined.  */
void orc_ce_from_substructures(const double A[9], const double* frac, int64_t N, double alpha_ew, const int nimg[3],
                               double kcut, double ke, const int32_t* site_class, const double* fixed_q,
                               const double* z, int32_t S, double* E_const, double* alpha, double* beta)
{
    int64_t nv = count_variable(site_class, N);
    int64_t* vidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int64_t v = 0;
    for (int64_t i = 0; i < N; ++i)
        if (site_class[i] >= 0) vidx[v++] = i;
    for (int64_t i = 0; i < N; ++i) q[i] = site_class[i] < 0 ? fixed_q[i] : 0.0;
    double e0 = orc_ewald_energy(A, frac, q, N, alpha_ew, nimg, kcut, ke);
    *E_const = e0;
    int64_t M = nv * S;
    for (int64_t a = 0; a < nv; ++a)
        for (int s = 0; s < S; ++s) {
            q[vidx[a]] = z[s];
            alpha[a * S + s] = orc_ewald_energy(A, frac, q, N, alpha_ew, nimg, kcut, ke) - e0;
            q[vidx[a]] = 0.0;
        }
    for (int64_t r = 0; r < M * M; ++r) beta[r] = 0.0;
    for (int64_t a = 0; a < nv; ++a)
        for (int64_t b = a + 1; b < nv; ++b)
            for (int s = 0; s < S; ++s)
                for (int t = 0; t < S; ++t) {
                    q[vidx[a]] = z[s];
                    q[vidx[b]] = z[t];
                    double e2 = orc_ewald_energy(A, frac, q, N, alpha_ew, nimg, kcut, ke);
                    q[vidx[a]] = 0.0;
                    q[vidx[b]] = 0.0;
                    beta[(a * S + s) * M + b * S + t] = e2 - alpha[a * S + s] - alpha[b * S + t] - e0;
                }
    free(vidx);
    free(q);
}

/* Eq. 2 objective for one configuration, through the binary vector x.      */
double orc_ce_energy(int64_t nv, int32_t S, double E_const, const double* alpha, const double* beta,
                     const int8_t* species_v)
{
    int64_t M = nv * S;
    uint8_t* x = (uint8_t*)calloc((size_t)(M > 0 ? M : 1), 1);
    for (int64_t a = 0; a < nv; ++a) x[a * S + species_v[a]] = 1;
    double e = E_const;
    for (int64_t r = 0; r < M; ++r) e += alpha[r] * x[r];
    for (int64_t r = 0; r < M; ++r)
        for (int64_t c = r + 1; c < M; ++c) e += beta[r * M + c] * (double)(x[r] * x[c]);
    free(x);
    return e;
}

/* ------------------------------------------------------------------------ */
/* Energy change of swapping the species at variable sites a and b          */
/* (SI, Monte Carlo: neighbours differ by a single atom swap).  With the    */
/* potential phi = J q (over all sites), d = q_b - q_a:                      */
/*   dE = 2 d (phi_a - phi_b) + d^2 (J_aa + J_bb - 2 J_ab).                  */
/* ia, ib are site indices into J (N x N).                                  */
/* ------------------------------------------------------------------------ */
double orc_delta_E(const double* J, int64_t N, const double* phi_site, int64_t ia, int64_t ib, double qa, double qb)
{
    double d = qb - qa;
    return 2.0 * d * (phi_site[ia] - phi_site[ib]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
}

/* ------------------------------------------------------------------------ */
/* Class bookkeeping shared by the heuristics.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t ncls;
    int64_t nv;
    int64_t* vsite;      /* nv: site index of variable site v                  */
    int32_t* vclass;     /* nv: class of variable site v                       */
    int64_t* cls_start;  /* ncls+1 offsets into cls_pos                        */
    int64_t* cls_pos;    /* variable-site indices grouped by class, ascending  */
    uint32_t* wprefix;   /* ncls: running sum of n_c (n_c - 1) over classes    */
    uint32_t wtotal;
    int32_t nmovable;    /* classes with at least two positions                */
    int32_t only_movable;/* the single movable class when nmovable == 1        */
} classes_t;

static classes_t make_classes(const int32_t* site_class, int64_t N)
{
    classes_t c;
    c.ncls = 0;
    for (int64_t i = 0; i < N; ++i)
        if (site_class[i] + 1 > c.ncls) c.ncls = site_class[i] + 1;
    c.nv = count_variable(site_class, N);
    c.vsite = (int64_t*)malloc(sizeof(int64_t) * (size_t)(c.nv + 1));
    c.vclass = (int32_t*)malloc(sizeof(int32_t) * (size_t)(c.nv + 1));
    c.cls_start = (int64_t*)calloc((size_t)c.ncls + 1, sizeof(int64_t));
    c.cls_pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(c.nv + 1));
    c.wprefix = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(c.ncls + 1));
    int64_t v = 0;
    for (int64_t i = 0; i < N; ++i)
        if (site_class[i] >= 0) {
            c.vsite[v] = i;
            c.vclass[v] = site_class[i];
            c.cls_start[site_class[i] + 1]++;
            v++;
        }
    for (int k = 0; k < c.ncls; ++k) c.cls_start[k + 1] += c.cls_start[k];
    int64_t* fill = (int64_t*)calloc((size_t)c.ncls + 1, sizeof(int64_t));
    for (int64_t w = 0; w < c.nv; ++w) {
        int k = c.vclass[w];
        c.cls_pos[c.cls_start[k] + fill[k]++] = w;
    }
    free(fill);
    uint64_t acc = 0;
    c.nmovable = 0;
    c.only_movable = -1;
    for (int k = 0; k < c.ncls; ++k) {
        uint64_t n = (uint64_t)(c.cls_start[k + 1] - c.cls_start[k]);
        if (n >= 2) {
            c.nmovable++;
            c.only_movable = k;
            acc += n * (n - 1);
        }
        c.wprefix[k] = (uint32_t)acc;
    }
    c.wtotal = (uint32_t)acc;
    return c;
}

static void free_classes(classes_t* c)
{
    free(c->vsite);
    free(c->vclass);
    free(c->cls_start);
    free(c->cls_pos);
    free(c->wprefix);
}

/* Pick the class of a swap: the only movable class, or one drawn with      */
/* weight n_c (n_c - 1), i.e. uniform over ordered position pairs.          */
static int pick_class(const classes_t* c, uint32_t x)
{
    if (c->nmovable == 1) return c->only_movable;
    uint32_t thr = draw_below(x, c->wtotal);
    for (int k = 0; k < c->ncls; ++k)
        if (c->wprefix[k] > thr) return k;
    return c->ncls - 1;
}

/* Ordered pair (a, b), a != b, uniform over positions of class k. */
static void pick_pair(const classes_t* c, int k, uint32_t xa, uint32_t xb, int64_t* va, int64_t* vb)
{
    uint32_t n = (uint32_t)(c->cls_start[k + 1] - c->cls_start[k]);
    uint32_t a = draw_below(xa, n);
    uint32_t bb = draw_below(xb, n - 1);
    uint32_t b = bb + (bb >= a);
    *va = c->cls_pos[c->cls_start[k] + a];
    *vb = c->cls_pos[c->cls_start[k] + b];
}

/* ------------------------------------------------------------------------ */
/* Random valid structures (SI, Random (R)): every class gets its multiset  */
/* of species (counts[k*S + s] of species s) in a uniformly random order by  */
/* a Fisher-Yates shuffle.  Draw t of class k for configuration b is word    */
/* t%4 of Philox(ctr = {t/4, b, k, 5}, key = seed).                          */
/* ------------------------------------------------------------------------ */
int orc_random_configs(int64_t N, const int32_t* site_class, int32_t S, const int32_t* counts, int64_t B,
                       uint64_t seed, int8_t* species)
{
    classes_t c = make_classes(site_class, N);
    int64_t nv = c.nv;
    int8_t* buf = (int8_t*)malloc((size_t)(nv + 1));
    for (int64_t b = 0; b < B; ++b) {
        int8_t* out = species + b * nv;
        for (int k = 0; k < c.ncls; ++k) {
            int64_t n = c.cls_start[k + 1] - c.cls_start[k];
            int64_t f = 0;
            for (int s = 0; s < S; ++s)
                for (int32_t r = 0; r < counts[k * S + s]; ++r) buf[f++] = (int8_t)s;
            if (f != n) {
                free(buf);
                free_classes(&c);
                return -1;
            }
            for (int64_t t = 0; t + 1 < n; ++t) {
                int64_t top = n - 1 - t;
                uint32_t x[4];
                philox_draw(seed, (uint32_t)(t >> 2), (uint32_t)b, (uint32_t)k, 5u, x);
                int64_t j = draw_below(x[t & 3], (uint32_t)(top + 1));
                int8_t tmp = buf[top];
                buf[top] = buf[j];
                buf[j] = tmp;
            }
            for (int64_t p = 0; p < n; ++p) out[c.cls_pos[c.cls_start[k] + p]] = buf[p];
        }
    }
    free(buf);
    free_classes(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Metropolis Monte Carlo with single-swap neighbours (SI, Monte Carlo):    */
/* accept with P = min[1, exp(-dE/kT)].  Chain c, step t (t counts from     */
/* step0), draws x = Philox(ctr = {t_lo, t_hi, c, 0}, key = seed):          */
/*   class: only movable class, else from Philox(ctr={t_lo,t_hi,c,1})[0];  */
/*   positions a = pos[x0*n >> 32], b = pos[b' + (b' >= a)], b' = x1*(n-1)>>32;*/
/*   u = ((x2 >> 5) * 2^26 + (x3 >> 6)) * 2^-53 in [0, 1).                   */
/* Equal species: a no-op trial.  Otherwise accept iff dE <= 1e-9 eV or      */
/* dE < -kT ln u, the event u < exp(-dE/kT) (u = 0 accepts; kT <= 0: dE <=  */
/* 1e-9 eV only); |dE| <= 1e-9 eV is read as dE = 0, since swaps related by */
/* symmetry give +-1e-14 eV under rounding.  On acceptance the species are  */
/* swapped, phi_w = fma(d, J[w,ia] - J[w,ib], phi_w) for every variable w,  */
/* and E += dE.  The best E seen (lower than every earlier one by more than  */
/* the 1e-9 eV tie) and its configuration are kept.  Returns the number of accepted swaps per chain in n_accept, and,   */
/* when E_trace (C x nsteps) is given, the energy before every step.         */
/* ------------------------------------------------------------------------ */
/* Temperature of step t: constant kT0, or with kT1 given the exponential    */
/* schedule kT0 (kT1/kT0)^(t/(total-1)) of simulated annealing (SI,          */
/* Simulated annealing: the temperature is lowered towards 0 during the run). */
static double step_kT(double kT0, const double* kT1, int64_t ch, uint64_t t, int64_t total)
{
    if (!kT1 || total <= 1) return kT0;
    return kT0 * exp(log(kT1[ch] / kT0) * ((double)t / (double)(total - 1)));
}

/* Stopping on a run without improvement (Section "Internal Fortran          */
/* Heuristics in GOAC": a run may end after a number of steps without         */
/* improvement).  With patience > 0 a chain stops after step t once           */
/* t - t_imp >= patience, t_imp being the last step whose acceptance lowered   */
/* E by more than 1e-9 eV below the energy at the previous such step (the     */
/* start, step0 - 1, counts as one).  Per-chain statistics (each nullable):    */
/* n_noop = proposals of two positions holding the same species; best_step =  */
/* the step at which the best E (lower than every earlier one by more than    */
/* 1e-9 eV) was reached (step0 - 1: the start); steps_done = steps run.       */
typedef struct {
    int64_t patience;
    int64_t* n_noop;
    int64_t* best_step;
    int64_t* steps_done;
} mc_extra;

static int mc_core(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                   int8_t* species, int64_t C, const double* kT, const double* kT1, int64_t total,
                   int64_t nsteps, uint64_t seed, uint64_t step0, double* E_out, double* bestE,
                   int8_t* best_species, int64_t* n_accept, double* E_trace, const mc_extra* ex);

int orc_mc_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
               int8_t* species, int64_t C, const double* kT, int64_t nsteps, uint64_t seed, uint64_t step0,
               double* E_out, double* bestE, int8_t* best_species, int64_t* n_accept, double* E_trace)
{
    return mc_core(J, N, site_class, fixed_q, z, species, C, kT, NULL, 0, nsteps, seed, step0, E_out, bestE,
                   best_species, n_accept, E_trace, NULL);
}

/* orc_mc_run with a patience (0: none) and the statistics described above. */
int orc_mc_run_ex(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                  int8_t* species, int64_t C, const double* kT, int64_t nsteps, uint64_t seed, uint64_t step0,
                  int64_t patience, double* E_out, double* bestE, int8_t* best_species, int64_t* n_accept,
                  int64_t* n_noop, int64_t* best_step, int64_t* steps_done)
{
    mc_extra ex = {patience, n_noop, best_step, steps_done};
    return mc_core(J, N, site_class, fixed_q, z, species, C, kT, NULL, 0, nsteps, seed, step0, E_out, bestE,
                   best_species, n_accept, NULL, &ex);
}

/* Simulated annealing: the Monte Carlo above with kT(t) = kT0 (kT1/kT0)^(t/(total-1)) per chain. */
int orc_sa_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
               int8_t* species, int64_t C, const double* kT0, const double* kT1, int64_t total, int64_t nsteps,
               uint64_t seed, uint64_t step0, double* E_out, double* bestE, int8_t* best_species, int64_t* n_accept)
{
    return mc_core(J, N, site_class, fixed_q, z, species, C, kT0, kT1, total, nsteps, seed, step0, E_out, bestE,
                   best_species, n_accept, NULL, NULL);
}

static int mc_core(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                   int8_t* species, int64_t C, const double* kT, const double* kT1, int64_t total,
                   int64_t nsteps, uint64_t seed, uint64_t step0, double* E_out, double* bestE,
                   int8_t* best_species, int64_t* n_accept, double* E_trace, const mc_extra* ex)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    if (cl.nmovable == 0) {
        free_classes(&cl);
        return -1;
    }
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* phi = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    for (int64_t ch = 0; ch < C; ++ch) {
        int8_t* sp = species + ch * nv;
        orc_config_charges(N, site_class, fixed_q, z, sp, q);
        double E = orc_qJq(J, q, N);
        for (int64_t w = 0; w < nv; ++w) {
            int64_t i = cl.vsite[w];
            double s = 0.0;
            for (int64_t j = 0; j < N; ++j) s += J[i * N + j] * q[j];
            phi[w] = s;
        }
        double best = E;
        if (best_species) memcpy(best_species + ch * nv, sp, (size_t)nv);
        int64_t nacc = 0, nnoop = 0, done = nsteps;
        int64_t t_best = (int64_t)step0 - 1, t_imp = (int64_t)step0 - 1;
        double E_imp = E;
        const int64_t patience = ex ? ex->patience : 0;
        for (int64_t s = 0; s < nsteps; ++s) {
            uint64_t t = step0 + (uint64_t)s;
            if (patience > 0 && (int64_t)t - 1 - t_imp >= patience) {   /* stopped after step t - 1 */
                done = s;
                break;
            }
            uint32_t x[4];
            philox_draw(seed, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)ch, 0u, x);
            int k;
            if (cl.nmovable == 1) k = cl.only_movable;
            else {
                uint32_t y[4];
                philox_draw(seed, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)ch, 1u, y);
                k = pick_class(&cl, y[0]);
            }
            int64_t va, vb;
            pick_pair(&cl, k, x[0], x[1], &va, &vb);
            int sa = sp[va], sb = sp[vb];
            if (E_trace) E_trace[ch * nsteps + s] = E;   /* energy before step s */
            if (sa == sb) {
                nnoop++;
                continue;
            }
            int64_t ia = cl.vsite[va], ib = cl.vsite[vb];
            double d = z[sb] - z[sa];
            double dE = 2.0 * d * (phi[va] - phi[vb]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
            double u = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6)) * (1.0 / 9007199254740992.0);
            const double kTt = step_kT(kT[ch], kT1, ch, t, total);
            int accept;
            /* Metropolis (SI, Monte Carlo): accept with probability min[1, exp(-dE/kT)],
               i.e. u < exp(-dE/kT), taken as the same event dE < -kT ln u */
            if (dE <= ORC_DE_ZERO) accept = 1;
            else if (kTt <= 0.0) accept = 0;
            else accept = u == 0.0 || dE < -kTt * log(u);
            if (!accept) continue;
            sp[va] = (int8_t)sb;
            sp[vb] = (int8_t)sa;
            /* phi_w += d (J_wa - J_wb), one rounding for the product and the sum */
            if (d != 0.0)
                for (int64_t w = 0; w < nv; ++w) {
                    int64_t i = cl.vsite[w];
                    phi[w] = fma(d, J[i * N + ia] - J[i * N + ib], phi[w]);
                }
            E = E + dE;
            nacc++;
            /* a new best must be lower by more than the 1e-9 eV tie: otherwise which of
               several symmetry-equivalent configurations is recorded follows rounding */
            if (E < best - ORC_DE_ZERO) {
                best = E;
                t_best = (int64_t)t;
                if (best_species) memcpy(best_species + ch * nv, sp, (size_t)nv);
            }
            if (E < E_imp - ORC_DE_ZERO) {
                E_imp = E;
                t_imp = (int64_t)t;
            }
        }
        if (E_out) E_out[ch] = E;
        if (bestE) bestE[ch] = best;
        if (n_accept) n_accept[ch] = nacc;
        if (ex && ex->n_noop) ex->n_noop[ch] = nnoop;
        if (ex && ex->best_step) ex->best_step[ch] = t_best;
        if (ex && ex->steps_done) ex->steps_done[ch] = done;
    }
    free(q);
    free(phi);
    free_classes(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The Metropolis rule of SI, Monte Carlo, taken literally: a twin of        */
/* mc_core that accepts iff dE <= 0, else iff u < exp(-dE/kT) (kT <= 0:      */
/* dE <= 0 only), and updates phi_w = phi_w + d (J_wa - J_wb) with the       */
/* product and the sum rounded separately.  Same draws, pair map and no-op   */
/* rule as mc_core.  It exists to show that mc_core's two readings (|dE| <=  */
/* 1e-9 eV counted as zero; the event u < exp(-dE/kT) tested as dE < -kT ln u */
/* with an fma update) take the paper's decisions on the tested workloads.   */
/* Per-chain diagnostics (each nullable): n_band = proposals with            */
/* 0 < dE <= 1e-9 eV (accepted outright by mc_core, drawn for here);         */
/* n_close = proposals with kT > 0 and |dE/kT + ln u| < 1e-9, where the two  */
/* forms of the Metropolis test could round to different decisions.         */
/* ------------------------------------------------------------------------ */
int orc_mc_run_literal(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q,
                       const double* z, int8_t* species, int64_t C, const double* kT, int64_t nsteps,
                       uint64_t seed, uint64_t step0, double* E_out, double* bestE, int64_t* n_accept,
                       int64_t* n_band, int64_t* n_close)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    if (cl.nmovable == 0) {
        free_classes(&cl);
        return -1;
    }
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* phi = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    for (int64_t ch = 0; ch < C; ++ch) {
        int8_t* sp = species + ch * nv;
        orc_config_charges(N, site_class, fixed_q, z, sp, q);
        double E = orc_qJq(J, q, N);
        for (int64_t w = 0; w < nv; ++w) {
            double acc = 0.0;
            for (int64_t j = 0; j < N; ++j) acc += J[cl.vsite[w] * N + j] * q[j];
            phi[w] = acc;
        }
        double best = E;
        int64_t nacc = 0, nband = 0, nclose = 0;
        for (int64_t s = 0; s < nsteps; ++s) {
            uint64_t t = step0 + (uint64_t)s;
            uint32_t x[4];
            philox_draw(seed, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)ch, 0u, x);
            int k = cl.only_movable;
            if (cl.nmovable != 1) {
                uint32_t y[4];
                philox_draw(seed, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)ch, 1u, y);
                k = pick_class(&cl, y[0]);
            }
            int64_t va, vb;
            pick_pair(&cl, k, x[0], x[1], &va, &vb);
            int sa = sp[va], sb = sp[vb];
            if (sa == sb) continue;
            int64_t ia = cl.vsite[va], ib = cl.vsite[vb];
            double d = z[sb] - z[sa];
            double dE = 2.0 * d * (phi[va] - phi[vb]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
            double u = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6)) * (1.0 / 9007199254740992.0);
            if (dE > 0.0 && dE <= 1e-9) nband++;
            if (kT[ch] > 0.0 && u > 0.0 && fabs(dE / kT[ch] + log(u)) < 1e-9) nclose++;
            int accept = dE <= 0.0 || (kT[ch] > 0.0 && u < exp(-dE / kT[ch]));
            if (!accept) continue;
            sp[va] = (int8_t)sb;
            sp[vb] = (int8_t)sa;
            for (int64_t w = 0; w < nv; ++w) {
                double dj = J[cl.vsite[w] * N + ia] - J[cl.vsite[w] * N + ib];
                double step = d * dj;
                phi[w] = phi[w] + step;
            }
            E = E + dE;
            nacc++;
            if (E < best - 1e-9) best = E;
        }
        if (E_out) E_out[ch] = E;
        if (bestE) bestE[ch] = best;
        if (n_accept) n_accept[ch] = nacc;
        if (n_band) n_band[ch] = nband;
        if (n_close) n_close[ch] = nclose;
    }
    free(q);
    free(phi);
    free_classes(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Genetic algorithm, one generation (SI, Genetic Algorithm; roulette wheel */
/* selection).  Population P x Nv with energies E.                          */
/*  1. Elitism: children 0..n_elite-1 are the n_elite lowest-E individuals, */
/*     ties broken by lower index.                                          */
/*  2. Roulette on integer fitness F_b = floor((Emax-E_b)/(Emax-Emin)*2^24)  */
/*     (all F_b = 1 when Emax == Emin).  A draw x (64 bit) selects the first */
/*     b whose running sum of F exceeds (x * F_total) >> 64.  Parents of      */
/*     child c in generation g: x_A = w0:w1, x_B = w2:w3 of                   */
/*     Philox(ctr = {0, g, c, 2}).                                           */
/*  3. Crossover, child = A.  For each variable site i (ascending) with       */
/*     child_i != B_i: j = the lowest site of i's class with child_j == B_i  */
/*     and B_j != B_i (one exists because class counts agree); draw k of the */
/*     child is word k%4 of Philox(ctr = {k/4, g, c, 3}); the swap i<->j is   */
/*     taken iff that word < 2^31 (probability 1/2).                          */
/*  4. Mutation: y = Philox(ctr = {0, g, c, 4}); if y0 < p_mut_u32 (and some */
/*     class has two positions) one swap                                      */
/*     of two positions of one class (class from y1, positions from y2, y3 as */
/*     in the Monte Carlo pair pick) is applied.                              */
/* parents_out (P x 2) and nswap_out (P x 2: swaps taken, candidate swaps)   */
/* record choices for testing; either may be NULL.  Children energies are computed afterwards (orc_score).      */
/* ------------------------------------------------------------------------ */
int orc_ga_generation(int64_t N, const int32_t* site_class, const int8_t* pop, const double* E, int64_t P,
                      int64_t n_elite, uint32_t p_mut_u32, uint32_t gen, uint64_t seed, int8_t* children,
                      int32_t* parents_out, int32_t* nswap_out)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    if (P <= 0 || n_elite < 0 || n_elite > P) {
        free_classes(&cl);
        return -1;
    }
    /* elitism: selection of the n_elite smallest by (E, index) */
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
    for (int64_t b = 0; b < P; ++b) order[b] = b;
    for (int64_t a = 0; a < n_elite; ++a) {       /* partial selection sort */
        int64_t m = a;
        for (int64_t b = a + 1; b < P; ++b) {
            int64_t ob = order[b], om = order[m];
            if (E[ob] < E[om] || (E[ob] == E[om] && ob < om)) m = b;
        }
        int64_t t = order[a];
        order[a] = order[m];
        order[m] = t;
    }
    for (int64_t a = 0; a < n_elite; ++a) {
        memcpy(children + a * nv, pop + order[a] * nv, (size_t)nv);
        if (parents_out) { parents_out[2 * a] = (int32_t)order[a]; parents_out[2 * a + 1] = (int32_t)order[a]; }
        if (nswap_out) { nswap_out[2 * a] = 0; nswap_out[2 * a + 1] = 0; }
    }
    free(order);

    /* roulette fitness */
    double emin = E[0], emax = E[0];
    for (int64_t b = 1; b < P; ++b) {
        if (E[b] < emin) emin = E[b];
        if (E[b] > emax) emax = E[b];
    }
    uint64_t* pre = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)P);
    uint64_t acc = 0;
    for (int64_t b = 0; b < P; ++b) {
        uint64_t f;
        if (emax > emin) f = (uint64_t)floor((emax - E[b]) / (emax - emin) * 16777216.0);
        else f = 1;
        acc += f;
        pre[b] = acc;
    }
    uint64_t ftot = acc;

    for (int64_t c = n_elite; c < P; ++c) {
        uint32_t x[4];
        philox_draw(seed, 0u, gen, (uint32_t)c, 2u, x);
        uint64_t xa = ((uint64_t)x[0] << 32) | x[1];
        uint64_t xb = ((uint64_t)x[2] << 32) | x[3];
        uint64_t ta = (uint64_t)(((unsigned __int128)xa * ftot) >> 64);
        uint64_t tb = (uint64_t)(((unsigned __int128)xb * ftot) >> 64);
        int64_t A = P - 1, Bp = P - 1;
        for (int64_t b = 0; b < P; ++b) if (pre[b] > ta) { A = b; break; }
        for (int64_t b = 0; b < P; ++b) if (pre[b] > tb) { Bp = b; break; }
        if (parents_out) { parents_out[2 * c] = (int32_t)A; parents_out[2 * c + 1] = (int32_t)Bp; }

        int8_t* ch = children + c * nv;
        const int8_t* pa = pop + A * nv;
        const int8_t* pb = pop + Bp * nv;
        memcpy(ch, pa, (size_t)nv);
        uint32_t k = 0;
        int32_t nsw = 0;
        uint32_t blk[4];
        for (int64_t i = 0; i < nv; ++i) {
            if (ch[i] == pb[i]) continue;
            int8_t want = pb[i];
            int cls = cl.vclass[i];
            int64_t j = -1;
            for (int64_t p = cl.cls_start[cls]; p < cl.cls_start[cls + 1]; ++p) {
                int64_t w = cl.cls_pos[p];
                if (ch[w] == want && pb[w] != want) { j = w; break; }
            }
            if (j < 0) { free(pre); free_classes(&cl); return -2; }
            if ((k & 3u) == 0) philox_draw(seed, k >> 2, gen, (uint32_t)c, 3u, blk);
            uint32_t w = blk[k & 3u];
            k++;
            if (w < 0x80000000u) {
                ch[j] = ch[i];
                ch[i] = want;
                nsw++;
            }
        }
        uint32_t y[4];
        philox_draw(seed, 0u, gen, (uint32_t)c, 4u, y);
        if (y[0] < p_mut_u32 && cl.nmovable > 0) {
            int kc = pick_class(&cl, y[1]);
            int64_t va, vb;
            pick_pair(&cl, kc, y[2], y[3], &va, &vb);
            int8_t t = ch[va];
            ch[va] = ch[vb];
            ch[vb] = t;
        }
        if (nswap_out) { nswap_out[2 * c] = nsw; nswap_out[2 * c + 1] = (int32_t)k; }
    }
    free(pre);
    free_classes(&cl);
    return 0;
}

/* Full GA run: init population -> n_gen generations (each followed by an   */
/* FP64 rescoring of every child).  Returns final population and energies.  */
int orc_ga_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
               int8_t* pop, double* E, int64_t P, int64_t n_gen, int64_t n_elite, uint32_t p_mut_u32,
               uint64_t seed, uint32_t gen0)
{
    int64_t nv = count_variable(site_class, N);
    int8_t* next = (int8_t*)malloc((size_t)(P * nv + 1));
    orc_score(J, N, site_class, fixed_q, z, pop, P, E);
    for (int64_t g = 0; g < n_gen; ++g) {
        int rc = orc_ga_generation(N, site_class, pop, E, P, n_elite, p_mut_u32, gen0 + (uint32_t)g, seed, next,
                                   NULL, NULL);
        if (rc) { free(next); return rc; }
        memcpy(pop, next, (size_t)(P * nv));
        orc_score(J, N, site_class, fixed_q, z, pop, P, E);
    }
    free(next);
    return 0;
}

/* GA run with the run-level stop of Section "Internal Fortran Heuristics in */
/* GOAC" (a run may end after a number of generations without improvement):  */
/* after generation g (1 ..) the population's lowest energy b_g is an        */
/* improvement when b_g < b_ref - 1e-9 eV, b_ref being the lowest energy at   */
/* the previous improvement (the initial population's at first); with        */
/* patience > 0 the run stops once `patience` generations in a row brought no */
/* improvement.  Outputs (nullable): generations run, the generation of the   */
/* last improvement (0: none) and whether patience stopped the run.           */
int orc_ga_run_ex(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                  int8_t* pop, double* E, int64_t P, int64_t n_gen, int64_t n_elite, uint32_t p_mut_u32,
                  uint64_t seed, uint32_t gen0, int64_t patience, int64_t* gens_out, int64_t* best_gen_out,
                  int32_t* stopped_out)
{
    int64_t nv = count_variable(site_class, N);
    int8_t* next = (int8_t*)malloc((size_t)(P * nv + 1));
    orc_score(J, N, site_class, fixed_q, z, pop, P, E);
    double b_ref = E[0];
    for (int64_t b = 1; b < P; ++b)
        if (E[b] < b_ref) b_ref = E[b];
    int64_t g = 0, stall = 0, best_gen = 0;
    int32_t stopped = 0;
    while (g < n_gen) {
        int rc = orc_ga_generation(N, site_class, pop, E, P, n_elite, p_mut_u32, gen0 + (uint32_t)g, seed, next,
                                   NULL, NULL);
        if (rc) { free(next); return rc; }
        memcpy(pop, next, (size_t)(P * nv));
        orc_score(J, N, site_class, fixed_q, z, pop, P, E);
        g++;
        double b_g = E[0];
        for (int64_t b = 1; b < P; ++b)
            if (E[b] < b_g) b_g = E[b];
        if (b_g < b_ref - ORC_DE_ZERO) {
            b_ref = b_g;
            stall = 0;
            best_gen = g;
        } else {
            stall++;
        }
        if (patience > 0 && stall >= patience) {
            stopped = 1;
            break;
        }
    }
    free(next);
    if (gens_out) *gens_out = g;
    if (best_gen_out) *best_gen_out = best_gen;
    if (stopped_out) *stopped_out = stopped;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Relaxed occupations (differentiable form).  logits L (Nv x S, per site,   */
/* species not allowed in the site's class are masked by allowed[k*S+s]=0); */
/* p = softmax over allowed species; q_v = sum_s p_vs z_s, q_f = fixed;      */
/*   E = q^T J q + lambda sum_{k,s allowed} (sum_{v in k} p_vs - n_ks)^2.    */
/* Gradient: g_vs = z_s (2 J q)_v + 2 lambda (sum_{w in k} p_ws - n_ks);     */
/*   dE/dL_vs = p_vs (g_vs - sum_t p_vt g_vt).                               */
/* ------------------------------------------------------------------------ */
double orc_energy_grad(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q,
                       const double* z, int32_t S, const int32_t* counts, const double* logits, double lambda,
                       double* dlogits)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    double* p = (double*)malloc(sizeof(double) * (size_t)(nv * S + 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* Jq = (double*)malloc(sizeof(double) * (size_t)N);
    double* colsum = (double*)calloc((size_t)(cl.ncls * S + 1), sizeof(double));
    for (int64_t v = 0; v < nv; ++v) {
        int k = cl.vclass[v];
        double m = -INFINITY;
        for (int s = 0; s < S; ++s)
            if (counts[k * S + s] > 0 && logits[v * S + s] > m) m = logits[v * S + s];
        double den = 0.0;
        for (int s = 0; s < S; ++s) {
            double e = counts[k * S + s] > 0 ? exp(logits[v * S + s] - m) : 0.0;
            p[v * S + s] = e;
            den += e;
        }
        for (int s = 0; s < S; ++s) {
            p[v * S + s] /= den;
            colsum[k * S + s] += p[v * S + s];
        }
    }
    {
        int64_t v = 0;
        for (int64_t i = 0; i < N; ++i) {
            if (site_class[i] < 0) q[i] = fixed_q[i];
            else {
                double s = 0.0;
                for (int t = 0; t < S; ++t) s += p[v * S + t] * z[t];
                q[i] = s;
                v++;
            }
        }
    }
    double E = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) s += J[i * N + j] * q[j];
        Jq[i] = s;
        E += q[i] * s;
    }
    for (int k = 0; k < cl.ncls; ++k)
        for (int s = 0; s < S; ++s)
            if (counts[k * S + s] > 0) {
                double r = colsum[k * S + s] - counts[k * S + s];
                E += lambda * r * r;
            }
    if (dlogits) {
        double* g = (double*)malloc(sizeof(double) * (size_t)(S + 1));
        for (int64_t v = 0; v < nv; ++v) {
            int k = cl.vclass[v];
            int64_t i = cl.vsite[v];
            double pg = 0.0;
            for (int s = 0; s < S; ++s) {
                g[s] = z[s] * 2.0 * Jq[i] + 2.0 * lambda * (colsum[k * S + s] - counts[k * S + s]);
                pg += p[v * S + s] * g[s];
            }
            for (int s = 0; s < S; ++s) dlogits[v * S + s] = counts[k * S + s] > 0 ? p[v * S + s] * (g[s] - pg) : 0.0;
        }
        free(g);
    }
    free(p);
    free(q);
    free(Jq);
    free(colsum);
    free_classes(&cl);
    return E;
}

/* Round relaxed occupations p (Nv x S, float) to a valid configuration:     */
/* per class, visit (site, species) pairs by p descending (ties: lower site, */
/* then lower species) and assign when the site is free and the species'     */
/* quota counts[k*S+s] is not used up.                                        */
typedef struct { float p; int64_t v; int32_t s; } pair_t;

static int pair_cmp(const void* a, const void* b)
{
    const pair_t* x = (const pair_t*)a;
    const pair_t* y = (const pair_t*)b;
    if (x->p > y->p) return -1;
    if (x->p < y->p) return 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return x->s < y->s ? -1 : (x->s > y->s);
}

int orc_round_to_counts(int64_t N, const int32_t* site_class, int32_t S, const int32_t* counts, const float* p,
                        int8_t* species)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(nv * S + 1));
    int32_t* left = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S + 1));
    uint8_t* done = (uint8_t*)calloc((size_t)nv + 1, 1);
    int rc = 0;
    for (int k = 0; k < cl.ncls && rc == 0; ++k) {
        int64_t m = 0;
        for (int64_t pp = cl.cls_start[k]; pp < cl.cls_start[k + 1]; ++pp) {
            int64_t v = cl.cls_pos[pp];
            for (int s = 0; s < S; ++s)
                if (counts[k * S + s] > 0) {
                    pr[m].p = p[v * S + s];
                    pr[m].v = v;
                    pr[m].s = s;
                    m++;
                }
        }
        qsort(pr, (size_t)m, sizeof(pair_t), pair_cmp);
        for (int s = 0; s < S; ++s) left[s] = counts[k * S + s];
        int64_t placed = 0;
        for (int64_t r = 0; r < m; ++r) {
            if (done[pr[r].v] || left[pr[r].s] == 0) continue;
            species[pr[r].v] = (int8_t)pr[r].s;
            done[pr[r].v] = 1;
            left[pr[r].s]--;
            placed++;
        }
        if (placed != cl.cls_start[k + 1] - cl.cls_start[k]) rc = -1;
    }
    free(pr);
    free(left);
    free(done);
    free_classes(&cl);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive enumeration (brute force) of all configurations of a tiny     */
/* problem: every class runs through all distinct orderings of its multiset */
/* (lexicographic next permutation).  Returns the number of configurations  */
/* (Eq. 1), the minimum energy, and up to max_argmin minimisers.             */
/* ------------------------------------------------------------------------ */
static int next_perm(int8_t* a, int64_t n)
{
    int64_t i = n - 2;
    while (i >= 0 && a[i] >= a[i + 1]) i--;
    if (i < 0) return 0;
    int64_t j = n - 1;
    while (a[j] <= a[i]) j--;
    int8_t t = a[i]; a[i] = a[j]; a[j] = t;
    for (int64_t l = i + 1, r = n - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

int64_t orc_enumerate(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                      int32_t S, const int32_t* counts, double tol, double* Emin, int8_t* argmin, int64_t max_argmin,
                      int64_t* n_argmin, double* all_E, int64_t max_all)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    int8_t** cur = (int8_t**)malloc(sizeof(int8_t*) * (size_t)(cl.ncls + 1));
    for (int k = 0; k < cl.ncls; ++k) {
        int64_t n = cl.cls_start[k + 1] - cl.cls_start[k];
        cur[k] = (int8_t*)malloc((size_t)(n + 1));
        int64_t f = 0;
        for (int s = 0; s < S; ++s)
            for (int32_t r = 0; r < counts[k * S + s]; ++r) cur[k][f++] = (int8_t)s;
    }
    int8_t* sp = (int8_t*)malloc((size_t)(nv + 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t total = 0, nmin = 0;
    double best = INFINITY;
    for (;;) {
        for (int k = 0; k < cl.ncls; ++k)
            for (int64_t p = cl.cls_start[k]; p < cl.cls_start[k + 1]; ++p) sp[cl.cls_pos[p]] = cur[k][p - cl.cls_start[k]];
        orc_config_charges(N, site_class, fixed_q, z, sp, q);
        double e = orc_qJq(J, q, N);
        if (all_E && total < max_all) all_E[total] = e;
        total++;
        if (e < best - tol) {
            best = e;
            nmin = 0;
        }
        if (fabs(e - best) <= tol) {
            if (argmin && nmin < max_argmin) memcpy(argmin + nmin * nv, sp, (size_t)nv);
            nmin++;
        }
        int k = 0;
        while (k < cl.ncls) {
            int64_t n = cl.cls_start[k + 1] - cl.cls_start[k];
            if (next_perm(cur[k], n)) break;
            /* wrapped: next_perm left it reversed-sorted; restore ascending */
            for (int64_t l = 0, r = n - 1; l < r; ++l, --r) { int8_t t = cur[k][l]; cur[k][l] = cur[k][r]; cur[k][r] = t; }
            k++;
        }
        if (k == cl.ncls) break;
    }
    *Emin = best;
    if (n_argmin) *n_argmin = nmin;
    for (int k = 0; k < cl.ncls; ++k) free(cur[k]);
    free(cur);
    free(sp);
    free(q);
    free_classes(&cl);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive enumeration for a problem whose only movable class holds two  */
/* species (every other site fixed): all C(n, k) placements of the k sites  */
/* of the second species among the class's n positions.  With q0 the        */
/* charges with species 0 everywhere in the class and delta = z1 - z0, the  */
/* energy of the set S of second-species positions is                       */
/*   E(S) = E0 + sum_{i in S} h_i + sum_{i<j in S} W_ij,                    */
/*   E0 = q0^T J q0,  h_i = 2 delta (J q0)_i + delta^2 J_ii,                */
/*   W_ij = 2 delta^2 J_ij,                                                 */
/* the quadratic form expanded in the occupation variables (Eq. 2 with two  */
/* species).  Positions are visited in order, depth first, include before  */
/* exclude; adding position i adds h_i + g_i with g = sum_{j in S} W_.j, and */
/* g is kept per depth (no undo, no drift).  Returns the number of          */
/* configurations, the minimum energy and the minimisers within tol (as     */
/* species vectors over the variable sites, up to max_argmin of them).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, k;
    const double* h;     /* n */
    const double* W;     /* n x n */
    double* g;           /* (k + 1) x n: field of the chosen set at each depth */
    int32_t* chosen;     /* k */
    double tol, best;
    int64_t total, nmin, max_argmin;
    int32_t* argsets;    /* max_argmin x k */
} enum2_t;

static void enum2_rec(enum2_t* st, int64_t pos, int64_t depth, double E)
{
    if (depth == st->k) {
        st->total++;
        if (E < st->best - st->tol) {
            st->best = E;
            st->nmin = 0;
        }
        if (fabs(E - st->best) <= st->tol) {
            if (st->nmin < st->max_argmin)
                memcpy(st->argsets + st->nmin * st->k, st->chosen, sizeof(int32_t) * (size_t)st->k);
            st->nmin++;
        }
        return;
    }
    if (st->n - pos < st->k - depth) return;
    /* include position pos */
    const double* g = st->g + depth * st->n;
    double* g2 = st->g + (depth + 1) * st->n;
    const double* Wp = st->W + pos * st->n;
    for (int64_t j = 0; j < st->n; ++j) g2[j] = g[j] + Wp[j];
    st->chosen[depth] = (int32_t)pos;
    enum2_rec(st, pos + 1, depth + 1, E + st->h[pos] + g[pos]);
    /* exclude it */
    enum2_rec(st, pos + 1, depth, E);
}

int64_t orc_enumerate_two_species(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q,
                                  const double* z, const int32_t* counts, double tol, double* Emin,
                                  int8_t* argmin, int64_t max_argmin, int64_t* n_argmin)
{
    classes_t cl = make_classes(site_class, N);
    if (cl.nmovable != 1 || cl.ncls != 1 || counts[0] + counts[1] != cl.nv) {
        free_classes(&cl);
        return -1;
    }
    const int64_t n = cl.nv, k = counts[1];
    int8_t* sp0 = (int8_t*)calloc((size_t)n + 1, 1);       /* species 0 everywhere */
    double* q0 = (double*)malloc(sizeof(double) * (size_t)N);
    orc_config_charges(N, site_class, fixed_q, z, sp0, q0);
    const double delta = z[1] - z[0];
    double* h = (double*)malloc(sizeof(double) * (size_t)n);
    double* W = (double*)malloc(sizeof(double) * (size_t)(n * n));
    for (int64_t a = 0; a < n; ++a) {
        const int64_t ia = cl.vsite[a];
        double jq = 0.0;
        for (int64_t j = 0; j < N; ++j) jq += J[ia * N + j] * q0[j];
        h[a] = 2.0 * delta * jq + delta * delta * J[ia * N + ia];
        for (int64_t b = 0; b < n; ++b) W[a * n + b] = a == b ? 0.0 : 2.0 * delta * delta * J[ia * N + cl.vsite[b]];
    }
    enum2_t st;
    st.n = n;
    st.k = k;
    st.h = h;
    st.W = W;
    st.g = (double*)calloc((size_t)((k + 1) * n), sizeof(double));
    st.chosen = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k + 1));
    st.tol = tol;
    st.best = INFINITY;
    st.total = 0;
    st.nmin = 0;
    st.max_argmin = max_argmin;
    st.argsets = (int32_t*)malloc(sizeof(int32_t) * (size_t)((max_argmin > 0 ? max_argmin : 1) * (k + 1)));
    enum2_rec(&st, 0, 0, orc_qJq(J, q0, N));
    *Emin = st.best;
    if (n_argmin) *n_argmin = st.nmin;
    const int64_t kept = st.nmin < max_argmin ? st.nmin : max_argmin;
    for (int64_t m = 0; m < kept && argmin; ++m) {
        int8_t* out = argmin + m * n;
        memset(out, 0, (size_t)n);
        for (int64_t t = 0; t < k; ++t) out[st.argsets[m * k + t]] = 1;
    }
    const int64_t total = st.total;
    free(st.g);
    free(st.chosen);
    free(st.argsets);
    free(h);
    free(W);
    free(q0);
    free(sp0);
    free_classes(&cl);
    return total;
}

/* Eq. 1: log10 C = sum_s [ log10 P_s! - sum_e log10 N_{s,e}! ].             */
double orc_log10_configurations(int32_t nsites, const int32_t* positions, int32_t nelem, const int32_t* n_se)
{
    double l = 0.0;
    for (int s = 0; s < nsites; ++s) {
        l += lgamma((double)positions[s] + 1.0);
        for (int e = 0; e < nelem; ++e) l -= lgamma((double)n_se[s * nelem + e] + 1.0);
    }
    return l / log(10.0);
}

/* ------------------------------------------------------------------------ */
/* Replica-exchange Monte Carlo (SI, Replica Exchange Monte Carlo): G groups */
/* of R chains (chain c = g R + slot) run Metropolis segments of              */
/* steps_per_round steps at their current temperatures; after round r the    */
/* neighbouring temperature ranks (k, k+1) with k = r%2, r%2 + 2, ... try to   */
/* exchange: with dE = E(chain at rank k) - E(chain at rank k+1), accept with */
/* P = min[1, exp(dE (1/kT_k - 1/kT_{k+1}))], u from words 0,1 of             */
/* Philox(ctr = {r, g, k, 6}).  An exchange swaps the two chains'             */
/* temperatures (equivalent to swapping configurations).  Segment r uses steps */
/* r*steps_per_round ...; perm[g R + k] = chain holding rank k.               */
/* ------------------------------------------------------------------------ */
int orc_remc_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                 int8_t* species, int64_t G, int64_t R, const double* kT_ladder, int64_t n_rounds,
                 int64_t steps_per_round, uint64_t seed, double* E_out, int32_t* perm, int64_t* n_exchanges)
{
    int64_t C = G * R;
    double* kT = (double*)malloc(sizeof(double) * (size_t)(C + 1));
    int64_t nex = 0;
    for (int64_t g = 0; g < G; ++g)
        for (int64_t k = 0; k < R; ++k) {
            perm[g * R + k] = (int32_t)(g * R + k);
            kT[g * R + k] = kT_ladder[k];
        }
    for (int64_t r = 0; r < n_rounds; ++r) {
        int rc = orc_mc_run(J, N, site_class, fixed_q, z, species, C, kT, steps_per_round, seed,
                            (uint64_t)(r * steps_per_round), E_out, NULL, NULL, NULL, NULL);
        if (rc) { free(kT); return rc; }
        for (int64_t g = 0; g < G; ++g)
            for (int64_t k = r % 2; k + 1 < R; k += 2) {
                int32_t ca = perm[g * R + k], cb = perm[g * R + k + 1];
                double dE = E_out[ca] - E_out[cb];
                double x = dE * (1.0 / kT_ladder[k] - 1.0 / kT_ladder[k + 1]);
                uint32_t w[4];
                philox_draw(seed, (uint32_t)r, (uint32_t)g, (uint32_t)k, 6u, w);
                double u = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * (1.0 / 9007199254740992.0);
                if (x >= 0.0 || u < exp(x)) {
                    perm[g * R + k] = cb;
                    perm[g * R + k + 1] = ca;
                    kT[ca] = kT_ladder[k + 1];
                    kT[cb] = kT_ladder[k];
                    nex++;
                }
            }
    }
    if (n_exchanges) *n_exchanges = nex;
    free(kT);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient descent over single-swap neighbours (SI, Gradient Descent: all  */
/* neighbours reachable by one swap are evaluated and the lowest is taken    */
/* until no neighbour is lower).  Each step: dE for every pair a < b of      */
/* variable sites of the same class holding different species; dmin = min;  */
/* if dmin < -1e-9 eV the step swaps the lowest pair (a, b) (lexicographic)  */
/* whose dE <= dmin + 1e-9 eV (energy ties within rounding resolve by index),*/
/* else the chain is at a local minimum.  At most max_steps steps.           */
/* ------------------------------------------------------------------------ */
int orc_gd_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
               int8_t* species, int64_t C, int64_t max_steps, double* E_out, int64_t* steps_out)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* phi = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    for (int64_t ch = 0; ch < C; ++ch) {
        int8_t* sp = species + ch * nv;
        orc_config_charges(N, site_class, fixed_q, z, sp, q);
        double E = orc_qJq(J, q, N);
        for (int64_t w = 0; w < nv; ++w) {
            int64_t i = cl.vsite[w];
            double s = 0.0;
            for (int64_t j = 0; j < N; ++j) s += J[i * N + j] * q[j];
            phi[w] = s;
        }
        int64_t steps = 0;
        while (steps < max_steps) {
            double dmin = INFINITY;
            for (int pass = 0; pass < 2; ++pass) {
                int64_t ba = -1, bb = -1;
                for (int64_t a = 0; a < nv && ba < 0; ++a)
                    for (int64_t b = a + 1; b < nv; ++b) {
                        if (cl.vclass[a] != cl.vclass[b] || sp[a] == sp[b]) continue;
                        int64_t ia = cl.vsite[a], ib = cl.vsite[b];
                        double d = z[sp[b]] - z[sp[a]];
                        double dE = 2.0 * d * (phi[a] - phi[b]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
                        if (pass == 0) {
                            if (dE < dmin) dmin = dE;
                        } else if (dE <= dmin + ORC_DE_ZERO) {
                            ba = a;
                            bb = b;
                            break;
                        }
                    }
                if (pass == 0 && !(dmin < -ORC_DE_ZERO)) goto done;
                if (pass == 1) {
                    int64_t ia = cl.vsite[ba], ib = cl.vsite[bb];
                    int sa = sp[ba], sb = sp[bb];
                    double d = z[sb] - z[sa];
                    double dE = 2.0 * d * (phi[ba] - phi[bb]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
                    sp[ba] = (int8_t)sb;
                    sp[bb] = (int8_t)sa;
                    for (int64_t w = 0; w < nv; ++w) {
                        int64_t i = cl.vsite[w];
                        phi[w] = phi[w] + d * (J[i * N + ia] - J[i * N + ib]);
                    }
                    E = E + dE;
                }
            }
            steps++;
        }
    done:
        if (E_out) E_out[ch] = E;
        if (steps_out) steps_out[ch] = steps;
    }
    free(q);
    free(phi);
    free_classes(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient descent with the SI, Gradient Descent rule taken literally: a     */
/* twin of orc_gd_run without the 1e-9 eV band.  Each step takes the lowest   */
/* dE over all same-class pairs a < b of different species; if it is < 0 the */
/* first pair (lexicographic) whose dE equals it exactly is swapped, else the */
/* configuration is a local minimum.  Used to show that the band of           */
/* orc_gd_run (ties within rounding resolved by index) changes no end state   */
/* of consequence on brute-forced cells.                                      */
/* ------------------------------------------------------------------------ */
int orc_gd_run_literal(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q,
                       const double* z, int8_t* species, int64_t C, int64_t max_steps, double* E_out,
                       int64_t* steps_out)
{
    classes_t cl = make_classes(site_class, N);
    int64_t nv = cl.nv;
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* phi = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    for (int64_t ch = 0; ch < C; ++ch) {
        int8_t* sp = species + ch * nv;
        orc_config_charges(N, site_class, fixed_q, z, sp, q);
        double E = orc_qJq(J, q, N);
        for (int64_t w = 0; w < nv; ++w) {
            double acc = 0.0;
            for (int64_t j = 0; j < N; ++j) acc += J[cl.vsite[w] * N + j] * q[j];
            phi[w] = acc;
        }
        int64_t steps = 0;
        for (; steps < max_steps; ++steps) {
            double dmin = 0.0;
            int64_t ba = -1, bb = -1;
            for (int64_t a = 0; a < nv; ++a)
                for (int64_t b = a + 1; b < nv; ++b) {
                    if (cl.vclass[a] != cl.vclass[b] || sp[a] == sp[b]) continue;
                    int64_t ia = cl.vsite[a], ib = cl.vsite[b];
                    double d = z[sp[b]] - z[sp[a]];
                    double dE = 2.0 * d * (phi[a] - phi[b]) + d * d * (J[ia * N + ia] + J[ib * N + ib] - 2.0 * J[ia * N + ib]);
                    if (dE < dmin) {
                        dmin = dE;
                        ba = a;
                        bb = b;
                    }
                }
            if (ba < 0) break;
            int64_t ia = cl.vsite[ba], ib = cl.vsite[bb];
            int sa = sp[ba], sb = sp[bb];
            double d = z[sb] - z[sa];
            sp[ba] = (int8_t)sb;
            sp[bb] = (int8_t)sa;
            for (int64_t w = 0; w < nv; ++w) {
                double dj = J[cl.vsite[w] * N + ia] - J[cl.vsite[w] * N + ib];
                double step = d * dj;
                phi[w] = phi[w] + step;
            }
            E = E + dmin;
        }
        if (E_out) E_out[ch] = E;
        if (steps_out) steps_out[ch] = steps;
    }
    free(q);
    free(phi);
    free_classes(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hybrid heuristic (SI, Hybrid Methods: REMC and GA are called alternately  */
/* and the best solutions are passed on).  P = G R configurations; cycle c:  */
/* REMC (n_rounds rounds of steps_per_round steps, key seed + 2c) on all P,  */
/* then n_gen GA generations (key seed + 2c + 1, generations numbered from   */
/* c n_gen, elitism keeps the best) starting from the REMC configurations;   */
/* the GA population (elites first) starts the next cycle's REMC.            */
/* ------------------------------------------------------------------------ */
int orc_hybrid_run(const double* J, int64_t N, const int32_t* site_class, const double* fixed_q, const double* z,
                   int8_t* species, int64_t G, int64_t R, const double* kT_ladder, int64_t n_cycles,
                   int64_t n_rounds, int64_t steps_per_round, int64_t n_gen, int64_t n_elite, uint32_t p_mut_u32,
                   uint64_t seed, double* E_out)
{
    int64_t P = G * R;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
    for (int64_t c = 0; c < n_cycles; ++c) {
        int rc = orc_remc_run(J, N, site_class, fixed_q, z, species, G, R, kT_ladder, n_rounds, steps_per_round,
                              seed + 2 * (uint64_t)c, E_out, perm, NULL);
        if (rc == 0)
            rc = orc_ga_run(J, N, site_class, fixed_q, z, species, E_out, P, n_gen, n_elite, p_mut_u32,
                            seed + 2 * (uint64_t)c + 1, (uint32_t)(c * n_gen));
        if (rc) { free(perm); return rc; }
    }
    free(perm);
    return 0;
}
