/*
 * FP64 CPU oracle for Grover-QAOA on 3-SAT (arXiv:2402.02585).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA path.
 *
 * Everything is written straight from the paper's definitions, in the
 * paper's order, with no blocking or fusion:
 *   - clause energy E_i and the problem Hamiltonian H_P (Section II.A, Eq. 1;
 *     satisfaction rule of Appendix B),
 *   - the G-QAOA state, phase e^{-i gamma H_P} then Grover mixer
 *     e^{-i beta |+><+|} per round (Section II.B, Eqs. 2-3),
 *   - the solution probability P = sum over solutions of |psi|^2 and the
 *     energy <H_P> (Eq. 4; Appendix B),
 *   - shots drawn by inverting the cumulative distribution of |psi|^2 in
 *     index order, from the Philox4x32-10 counter-based generator (Salmon,
 *     Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *     SC 2011), written from that paper's definition.
 *
 * Conventions (readings of the paper):
 *   - bit j of the assignment index z is Boolean variable j (value 1 = true);
 *   - literals are DIMACS integers: +(v+1) is x_v, -(v+1) is NOT x_v.
 *
 * Complex numbers are stored interleaved (re, im) as double[2*N].
 * OpenMP parallel loops are used for speed on large n; they change only the
 * order of FP64 additions in reductions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- problem Hamiltonian -------------------------------------------- */

/* Appendix B: an assignment satisfies literal x when tau(x)=1 and literal
 * NOT x when tau(x)=0; it satisfies a clause when it satisfies at least one
 * of its literals. Eq. 1: E_i = 1 exactly when clause i is not satisfied.
 * H_P(z) = sum_i E_i is the number of unsatisfied clauses. */
int oracle_cost_at(const int32_t *lits, int m, uint64_t z)
{
    int unsat = 0;
    for (int i = 0; i < m; ++i) {
        int satisfied = 0;
        for (int j = 0; j < 3; ++j) {
            int32_t lit = lits[3 * i + j];
            int var = (lit > 0 ? lit : -lit) - 1;
            int value = (int)((z >> var) & 1u);
            if (lit > 0 && value == 1) satisfied = 1;
            if (lit < 0 && value == 0) satisfied = 1;
        }
        if (!satisfied) unsat += 1;
    }
    return unsat;
}

/* Cost table C(z) for all z in [0, 2^n) and its histogram h[c] = #{z: C(z)=c}
 * (the energy-manifold counts of Appendix C). Returns 0, or -1 on bad
 * arguments (n outside 1..34, m outside 0..255, a literal out of range). */
int oracle_cost_table(const int32_t *lits, int n, int m, uint8_t *cost, uint64_t *hist)
{
    if (n < 1 || n > 34 || m < 0 || m > 255) return -1;
    for (int i = 0; i < 3 * m; ++i) {
        int32_t lit = lits[i];
        if (lit == 0 || lit > n || lit < -n) return -1;
    }
    uint64_t N = (uint64_t)1 << n;
    memset(hist, 0, sizeof(uint64_t) * (size_t)(m + 1));
#pragma omp parallel
    {
        uint64_t local[256];
        memset(local, 0, sizeof(local));
#pragma omp for schedule(static)
        for (int64_t z = 0; z < (int64_t)N; ++z) {
            int c = oracle_cost_at(lits, m, (uint64_t)z);
            if (cost) cost[z] = (uint8_t)c;
            local[c] += 1;
        }
#pragma omp critical
        for (int c = 0; c <= m; ++c) hist[c] += local[c];
    }
    return 0;
}

/* ---- G-QAOA evolution (Eqs. 2-3) --------------------------------------- */

/* |+> = 2^{-n/2} sum_z |z>. */
void oracle_plus_state(int n, double *psi)
{
    uint64_t N = (uint64_t)1 << n;
    double amp = 1.0 / sqrt((double)N);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        psi[2 * z] = amp;
        psi[2 * z + 1] = 0.0;
    }
}

/* One phase step psi <- e^{-i gamma H_P} psi. H_P is diagonal with entries
 * C(z), so each amplitude is multiplied by e^{-i gamma C(z)}. The m+1
 * possible factors are formed once. */
void oracle_apply_phase(const uint8_t *cost, int n, double gamma, double *psi)
{
    uint64_t N = (uint64_t)1 << n;
    double fre[256], fim[256];
    for (int c = 0; c < 256; ++c) {
        fre[c] = cos(gamma * (double)c);
        fim[c] = -sin(gamma * (double)c);
    }
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        int c = cost[z];
        double re = psi[2 * z], im = psi[2 * z + 1];
        psi[2 * z] = fre[c] * re - fim[c] * im;
        psi[2 * z + 1] = fre[c] * im + fim[c] * re;
    }
}

/* One mixer step psi <- e^{-i beta H_M} psi with H_M = |+><+| (Eq. 2).
 * H_M is a rank-1 projector, so e^{-i beta H_M} = 1 + (e^{-i beta} - 1)|+><+|
 * and |+><+|psi> = (2^{-n} sum_z psi(z)) * (1, ..., 1). */
void oracle_apply_mixer(int n, double beta, double *psi)
{
    uint64_t N = (uint64_t)1 << n;
    double sre = 0.0, sim = 0.0;
#pragma omp parallel for reduction(+ : sre, sim) schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        sre += psi[2 * z];
        sim += psi[2 * z + 1];
    }
    double mre = sre / (double)N, mim = sim / (double)N;
    double cre = cos(beta) - 1.0, cim = -sin(beta); /* e^{-i beta} - 1 */
    double are = cre * mre - cim * mim, aim = cre * mim + cim * mre;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        psi[2 * z] += are;
        psi[2 * z + 1] += aim;
    }
}

/* Solution probability and energy of a state (Eq. 4; Appendix B):
 * out[0] = sum_{z: C(z)=0} |psi(z)|^2, out[1] = sum_z C(z)|psi(z)|^2,
 * out[2] = sum_z |psi(z)|^2. */
void oracle_readout(const double *psi, const uint8_t *cost, int n, double *out)
{
    uint64_t N = (uint64_t)1 << n;
    double p0 = 0.0, e = 0.0, norm = 0.0;
#pragma omp parallel for reduction(+ : p0, e, norm) schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        double w = psi[2 * z] * psi[2 * z] + psi[2 * z + 1] * psi[2 * z + 1];
        norm += w;
        e += (double)cost[z] * w;
        if (cost[z] == 0) p0 += w;
    }
    out[0] = p0;
    out[1] = e;
    out[2] = norm;
}

/* Eq. 3: |beta, gamma> = e^{-i b_p H_M} e^{-i g_p H_P} ... e^{-i b_1 H_M} e^{-i g_1 H_P} |+>.
 * If from_plus is nonzero psi is first set to |+>; otherwise psi holds the
 * initial state. trace (may be NULL) receives P after each round. */
void oracle_evolve(const uint8_t *cost, int n, const double *gammas, const double *betas,
                   int p, double *psi, int from_plus, double *trace)
{
    if (from_plus) oracle_plus_state(n, psi);
    for (int k = 0; k < p; ++k) {
        oracle_apply_phase(cost, n, gammas[k], psi);
        oracle_apply_mixer(n, betas[k], psi);
        if (trace) {
            double r[3];
            oracle_readout(psi, cost, n, r);
            trace[k] = r[0];
        }
    }
}

/* ---- Philox4x32-10 (Salmon et al., SC 2011) ---------------------------- */

/* One round: two 32x32->64 products of the counter's even words with the
 * round multipliers; the high halves are xored with the odd words and the
 * key, and the words are permuted. Ten rounds, the key bumped by the Weyl
 * constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in [0,1) for shot s of a stream: Philox4x32-10 with
 * counter (s_lo, s_hi, 0, 0) and key (seed_lo, seed_hi); the top 53 bits of
 * the 64-bit word (out1:out0) scaled by 2^-53. */
double oracle_shot_uniform(uint64_t seed, uint64_t shot)
{
    uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    uint64_t x = ((uint64_t)r[1] << 32) | (uint64_t)r[0];
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* Shots z ~ |psi(z)|^2 by inversion of the cumulative distribution in index
 * order: shot s is the smallest z with CDF(z) > u_s * CDF(N-1), CDF(z) the
 * sum of |psi|^2 up to and including z. The running sum carries the rounding
 * error of every addition in a second word (Neumaier's compensated
 * summation), so each CDF(z) is within a few units in the last place of the
 * exact sum of the FP64 weights however many terms precede it; a plain
 * running sum would drift by up to N rounding errors over 2^n terms. If
 * cdf_out is not NULL it receives the CDF. Returns 0, or -1 if the state has
 * zero norm. */
int oracle_sample(const double *psi, int n, uint64_t seed, int64_t shots, uint32_t *out,
                  double *cdf_out)
{
    uint64_t N = (uint64_t)1 << n;
    double *cdf = cdf_out ? cdf_out : (double *)malloc(sizeof(double) * N);
    if (!cdf) return -1;
    double run = 0.0, carry = 0.0;
    for (uint64_t z = 0; z < N; ++z) {
        double w = psi[2 * z] * psi[2 * z] + psi[2 * z + 1] * psi[2 * z + 1];
        double t = run + w;
        if (fabs(run) >= fabs(w))
            carry += (run - t) + w;  /* the low part of run + w lost in t */
        else
            carry += (w - t) + run;
        run = t;
        cdf[z] = run + carry;
    }
    double total = cdf[N - 1];
    int status = 0;
    if (!(total > 0.0)) {
        status = -1;
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < shots; ++s) {
            double t = oracle_shot_uniform(seed, (uint64_t)s) * total;
            uint64_t lo = 0, hi = N - 1; /* smallest z with cdf[z] > t */
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (cdf[mid] > t) hi = mid; else lo = mid + 1;
            }
            out[s] = (uint32_t)lo;
        }
    }
    if (!cdf_out) free(cdf);
    return status;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by the OpenMP loops from now on (timing on one core). */
void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
