/*
 * rbe_oracle.c -- plain, slow FP64 CPU oracle for the random batch Ewald (RBE)
 * method of Jin, Li, Xu and Zhao, "A random batch Ewald method for particle
 * systems with Coulomb interactions" (arXiv:2010.01559).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) never calls it, and the two share no code: this file has
 * its own Philox, its own sampling table, its own Ewald sums.
 *
 * Everything is double precision, straight loops, no blocking and no fusion
 * beyond what the formulas state; OpenMP only splits the outer loop over
 * particles (each thread owns whole rows, so results do not depend on the
 * thread count).
 *
 * Conventions (Sec. 2):
 *   r_ij = r_j - r_i, V = L^3, k = 2*pi*m/L, m in Z^3.
 *   lB multiplies every Coulomb term (Sec. 4.1: eps = 1/4pi gives phi = q/r,
 *   i.e. lB = 1; Sec. 4.2 scales by the Bjerrum length).
 *
 * Every function below is pinned by tests against closed forms, textbook
 * values or brute force (NaCl Madelung constant, alpha-independence of the
 * Ewald energy, direct image sums, exact expectation and variance of the
 * estimator, finite differences, published Philox vectors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,         */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Written from the   */
/* published description: 10 rounds of two 32x32->64 multiplies with the     */
/* round multipliers, the key bumped by the two Weyl constants between rounds.*/
/* ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
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

/* ------------------------------------------------------------------------- */
/* Sampling of k (Sec. 3.1, Eq. probexpression and the per-axis marginal      */
/* P(m) ~ exp(-(2 pi m / L)^2 / (4 alpha)) = exp(-pi^2 m^2 / (alpha L^2))).   */
/*                                                                           */
/* The per-axis weights are tabulated for |m| <= M with                      */
/*   M = ceil( sqrt(alpha L^2 ln 2^64) / pi ),                               */
/* so the weight left out is below 2^-64 of the largest one.  H is the       */
/* direct sum of the tabulated weights (Eq. psf, first form), S = H^3 - 1    */
/* (Eq. S).  The cumulative table holds floor(2^32 * CDF) so that a uniform  */
/* 32-bit word maps to m by integer comparison only.                         */
/* ------------------------------------------------------------------------- */
int orc_axis_M(double alpha, double L)
{
    double x = sqrt(alpha * L * L * (64.0 * log(2.0))) / M_PI;
    return (int)ceil(x);
}

/* T has 2M+1 entries; T[2M] = 2^32.  Returns H (= Z, the normaliser). */
double orc_axis_table(double alpha, double L, int M, uint64_t *T)
{
    const double a = (M_PI * M_PI) / (alpha * L * L);
    const int n = 2 * M + 1;
    double Z = 0.0;
    for (int j = 0; j < n; ++j) {
        long mm = (long)(j - M) * (long)(j - M);
        Z += exp(-(a * (double)mm));
    }
    double cum = 0.0;
    for (int j = 0; j < n; ++j) {
        long mm = (long)(j - M) * (long)(j - M);
        cum += exp(-(a * (double)mm));
        if (j == n - 1) {
            T[j] = 4294967296ull;
        } else {
            double f = floor((cum / Z) * 4294967296.0);
            if (f > 4294967295.0) f = 4294967295.0;
            T[j] = (uint64_t)f;
        }
    }
    return Z;
}

/* Smallest j with w < T[j], minus M: an integer inverse-CDF lookup. */
static int orc_axis_lookup(const uint64_t *T, int M, uint32_t w)
{
    int j = 0;
    while ((uint64_t)w >= T[j]) ++j;
    return j - M;
}

/* Draw P i.i.d. samples m in Z^3 \ {0} from P_k (Eq. probexpression) for one
 * (seed, stream, step).  Sample l, attempt a uses
 *   Philox(key = (seed_lo, seed_hi), ctr = (l, a, step_lo, (stream << 8) | 1))
 * and words 0..2 give m_x, m_y, m_z.  A draw of (0,0,0) is discarded (Sec.
 * 3.1) and redrawn with attempt a+1.  m is P x 3, attempts (nullable) P.
 * Returns 0, or 1 if some sample needed more than 32 attempts. */
int orc_sample_k(double alpha, double L, uint64_t seed, uint32_t stream, uint64_t step,
                 int P, int32_t *m, int32_t *attempts)
{
    int M = orc_axis_M(alpha, L);
    uint64_t *T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    orc_axis_table(alpha, L, M, T);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int bad = 0;
    for (int l = 0; l < P; ++l) {
        int a = 0, ok = 0;
        int mx = 0, my = 0, mz = 0;
        for (a = 0; a < 32; ++a) {
            uint32_t ctr[4] = {(uint32_t)l, (uint32_t)a, (uint32_t)step, (stream << 8) | 0x01u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            mx = orc_axis_lookup(T, M, w[0]);
            my = orc_axis_lookup(T, M, w[1]);
            mz = orc_axis_lookup(T, M, w[2]);
            if (mx != 0 || my != 0 || mz != 0) { ok = 1; break; }
        }
        if (!ok) { bad = 1; mx = my = mz = 0; }
        m[3 * l + 0] = mx; m[3 * l + 1] = my; m[3 * l + 2] = mz;
        if (attempts) attempts[l] = a + 1;
    }
    free(T);
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Fourier part of the Ewald sum for one explicit list of wave vectors.      */
/*                                                                           */
/* Each wave vector l carries a weight c_l and contributes                   */
/*   energy   c_l * (2 pi / (V k^2)) |rho(k)|^2                              */
/*   force    -c_l * (4 pi q_i k / (V k^2)) Im(e^{-i k.r_i} rho(k))          */
/*   dE/dq_i  c_l * (4 pi / (V k^2)) Re(e^{-i k.r_i} rho(k))                 */
/* with rho(k) = sum_j q_j e^{i k.r_j} (Sec. 2).  Full Ewald takes           */
/* c = exp(-k^2 / 4 alpha) over all k != 0 in a cube (Eq. force, first       */
/* term); RBE takes c = S / P for P sampled k (Eq. rbmapprox).  The self     */
/* term -sqrt(alpha/pi) sum q^2 (Sec. 2) and the neutralising-background     */
/* term -pi (sum q)^2 / (2 V alpha) (zero for a neutral system) are added    */
/* to the energy, and their q-derivatives to dE/dq.  All scaled by lB.       */
/*                                                                           */
/* Forces and dE/dq are computed only for the nsub particles listed in sub   */
/* (all particles if sub is NULL); rho always runs over all N.               */
/* ------------------------------------------------------------------------- */
static void orc_fourier_weighted(int N, const double *pos, const double *q, double L,
                                 double alpha, double lB, int K, const int32_t *m,
                                 const double *c, int nsub, const int *sub,
                                 double *F, double *phi, double *E, double *rho_out)
{
    const double V = L * L * L;
    const double twopi_L = 2.0 * M_PI / L;
    double *rre = (double *)calloc((size_t)K, sizeof(double));
    double *rim = (double *)calloc((size_t)K, sizeof(double));

    /* rho(k_l) = sum_j q_j (cos(k.r_j) + i sin(k.r_j)) */
    #pragma omp parallel for schedule(static)
    for (int l = 0; l < K; ++l) {
        double kx = twopi_L * m[3 * l + 0], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < N; ++j) {
            double th = kx * pos[3 * j + 0] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
            sr += q[j] * cos(th);
            si += q[j] * sin(th);
        }
        rre[l] = sr;
        rim[l] = si;
    }

    double qsum = 0.0, q2sum = 0.0;
    for (int j = 0; j < N; ++j) { qsum += q[j]; q2sum += q[j] * q[j]; }

    if (E) {
        double e = 0.0;
        for (int l = 0; l < K; ++l) {
            double kx = twopi_L * m[3 * l + 0], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
            double k2 = kx * kx + ky * ky + kz * kz;
            e += c[l] * (2.0 * M_PI / (V * k2)) * (rre[l] * rre[l] + rim[l] * rim[l]);
        }
        e -= sqrt(alpha / M_PI) * q2sum;
        e -= M_PI * qsum * qsum / (2.0 * V * alpha);
        E[0] = lB * e;
    }
    if (rho_out) {
        for (int l = 0; l < K; ++l) { rho_out[2 * l] = rre[l]; rho_out[2 * l + 1] = rim[l]; }
    }

    int n_out = sub ? nsub : N;
    #pragma omp parallel for schedule(static)
    for (int t = 0; t < n_out; ++t) {
        int i = sub ? sub[t] : t;
        double fx = 0.0, fy = 0.0, fz = 0.0, ph = 0.0;
        for (int l = 0; l < K; ++l) {
            double kx = twopi_L * m[3 * l + 0], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
            double k2 = kx * kx + ky * ky + kz * kz;
            double th = kx * pos[3 * i + 0] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
            double ct = cos(th), st = sin(th);
            /* e^{-i th} rho = (ct - i st)(re + i im) */
            double im_part = ct * rim[l] - st * rre[l];
            double re_part = ct * rre[l] + st * rim[l];
            double g = c[l] * 4.0 * M_PI / (V * k2);
            fx -= g * q[i] * kx * im_part;
            fy -= g * q[i] * ky * im_part;
            fz -= g * q[i] * kz * im_part;
            ph += g * re_part;
        }
        if (F) {
            F[3 * t + 0] = lB * fx; F[3 * t + 1] = lB * fy; F[3 * t + 2] = lB * fz;
        }
        if (phi) {
            ph -= 2.0 * sqrt(alpha / M_PI) * q[i];
            ph -= M_PI * qsum / (V * alpha);
            phi[t] = lB * ph;
        }
    }
    free(rre);
    free(rim);
}

/* Full (deterministic) Ewald Fourier part over 0 < |m|_inf <= mmax (Sec. 2,
 * U_1 and the first term of Eq. force). */
void orc_ewald_fourier(int N, const double *pos, const double *q, double L, double alpha,
                       double lB, int mmax, int nsub, const int *sub,
                       double *F, double *phi, double *E)
{
    int side = 2 * mmax + 1;
    int K = side * side * side - 1;
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)K);
    double *c = (double *)malloc(sizeof(double) * (size_t)K);
    int t = 0;
    for (int a = -mmax; a <= mmax; ++a)
        for (int b = -mmax; b <= mmax; ++b)
            for (int d = -mmax; d <= mmax; ++d) {
                if (a == 0 && b == 0 && d == 0) continue;
                m[3 * t] = a; m[3 * t + 1] = b; m[3 * t + 2] = d;
                double k2 = (2.0 * M_PI / L) * (2.0 * M_PI / L) * (double)(a * a + b * b + d * d);
                c[t] = exp(-k2 / (4.0 * alpha));
                ++t;
            }
    orc_fourier_weighted(N, pos, q, L, alpha, lB, K, m, c, nsub, sub, F, phi, E, NULL);
    free(m);
    free(c);
}

/* RBE Fourier estimator for a given batch of P wave vectors (Eq. rbmapprox):
 * every sampled k carries the weight S/P.  The energy returned is the
 * frozen-batch estimator whose exact gradient is -F. */
void orc_rbe_fourier(int N, const double *pos, const double *q, double L, double alpha,
                     double lB, double S, int P, const int32_t *m, int nsub, const int *sub,
                     double *F, double *phi, double *E, double *rho)
{
    double *c = (double *)malloc(sizeof(double) * (size_t)P);
    for (int l = 0; l < P; ++l) c[l] = S / (double)P;
    orc_fourier_weighted(N, pos, q, L, alpha, lB, P, m, c, nsub, sub, F, phi, E, rho);
    free(c);
}

/* Exact single-k RBE force (P = 1, weight S) for every particle: used by the
 * tests to form the expectation sum_k P_k F*(k) exactly. */
void orc_rbe_single_k_force(int N, const double *pos, const double *q, double L, double alpha,
                            double lB, double S, const int32_t *m1, double *F)
{
    double c = S;
    orc_fourier_weighted(N, pos, q, L, alpha, lB, 1, m1, &c, 0, NULL, F, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------- */
/* Real-space part (Sec. 2, U_2 truncated at r_c, and the second term of     */
/* Eq. force) and the shifted Lennard-Jones potential (Eq. Ljpotential with  */
/* r_off = 0, cut at lj_rcut and shifted to zero there).  The cutoff is at   */
/* most L/2, so the minimum image is the only image within it.  All pairs.   */
/*                                                                           */
/* Outputs (all nullable): Fc, Flj (nsub x 3), phi (nsub), E[0] = Coulomb    */
/* real-space energy, E[1] = LJ energy (over all particles).                 */
/* ------------------------------------------------------------------------- */
void orc_real_space(int N, const double *pos, const double *q, double L, double alpha,
                    double r_c, double lB, double lj_eps, double lj_sigma, double lj_rcut,
                    int nsub, const int *sub, double *Fc, double *Flj, double *phi, double *E)
{
    const double sa = sqrt(alpha);
    int n_out = sub ? nsub : N;
    double ec = 0.0, elj = 0.0;
    double vshift = 0.0;
    if (lj_eps != 0.0) {
        double sr6 = pow(lj_sigma / lj_rcut, 6.0);
        vshift = -4.0 * lj_eps * (sr6 * sr6 - sr6);
    }
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : ec, elj)
    for (int t = 0; t < n_out; ++t) {
        int i = sub ? sub[t] : t;
        double fcx = 0, fcy = 0, fcz = 0, flx = 0, fly = 0, flz = 0, ph = 0;
        double eci = 0.0, elji = 0.0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3];
            for (int a = 0; a < 3; ++a) {
                double x = pos[3 * j + a] - pos[3 * i + a];   /* r_ij = r_j - r_i */
                x -= L * nearbyint(x / L);
                d[a] = x;
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            if (r < r_c) {
                double erfc_r = erfc(sa * r);
                double G = erfc_r / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r);
                /* F_i,2 = -q_i q_j G(r) r_ij / r */
                double s = -lB * q[i] * q[j] * G / r;
                fcx += s * d[0]; fcy += s * d[1]; fcz += s * d[2];
                ph += lB * q[j] * erfc_r / r;
                eci += 0.5 * lB * q[i] * q[j] * erfc_r / r;
            }
            if (lj_eps != 0.0 && r < lj_rcut) {
                double sr2 = (lj_sigma * lj_sigma) / r2;
                double sr6 = sr2 * sr2 * sr2;
                /* -dV/dr = 24 eps (2 (s/r)^12 - (s/r)^6) / r, directed along -r_ij */
                double mag = 24.0 * lj_eps * (2.0 * sr6 * sr6 - sr6) / r;
                flx -= mag * d[0] / r; fly -= mag * d[1] / r; flz -= mag * d[2] / r;
                elji += 0.5 * (4.0 * lj_eps * (sr6 * sr6 - sr6) + vshift);
            }
        }
        if (Fc) { Fc[3 * t] = fcx; Fc[3 * t + 1] = fcy; Fc[3 * t + 2] = fcz; }
        if (Flj) { Flj[3 * t] = flx; Flj[3 * t + 1] = fly; Flj[3 * t + 2] = flz; }
        if (phi) phi[t] = ph;
        ec += eci;
        elj += elji;
    }
    if (E) { E[0] = ec; E[1] = elj; }
}

/* ------------------------------------------------------------------------- */
/* Brute-force image sum (Eq. energy): U = 1/2 sum'_n sum_ij q_i q_j /       */
/* |r_ij + n L| over the cube |n|_inf <= R, n = 0 excluded for i = j.  For a  */
/* neutral cell this cube-ordered sum tends to the tin-foil Ewald energy     */
/* plus the surface term (2 pi / 3V) |sum_i q_i r_i|^2.  Unscaled (lB = 1).  */
/* ------------------------------------------------------------------------- */
double orc_brute_images(int N, const double *pos, const double *q, double L, int R)
{
    double U = 0.0;
    #pragma omp parallel for schedule(static) reduction(+ : U) collapse(2)
    for (int a = -R; a <= R; ++a)
        for (int b = -R; b <= R; ++b) {
            double u = 0.0;
            for (int c = -R; c <= R; ++c)
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double dx = pos[3 * j] - pos[3 * i] + a * L;
                        double dy = pos[3 * j + 1] - pos[3 * i + 1] + b * L;
                        double dz = pos[3 * j + 2] - pos[3 * i + 2] + c * L;
                        u += q[i] * q[j] / sqrt(dx * dx + dy * dy + dz * dz);
                    }
            U += u;
        }
    return 0.5 * U;
}

/* ------------------------------------------------------------------------- */
/* Proposition 1 (Sec. 3.2, Eq. varianceforce): exact E|chi_i|^2 of the RBE  */
/* Fourier force with batch size P, using every k with 0 < |m|_inf <= mmax,  */
/*   E|chi_i|^2 = (1/P) ( sum_k (4 pi q_i)^2 S / (V^2 k^2) e^{-k^2/4alpha}    */
/*                        |Im(e^{-ik.r_i} rho(k))|^2 - |F_i,1|^2 ),          */
/* with lB^2 applied.  F1 (N x 3, nullable) receives F_i,1.                  */
/* ------------------------------------------------------------------------- */
void orc_fourier_variance(int N, const double *pos, const double *q, double L, double alpha,
                          double lB, double S, int mmax, int P, double *var, double *F1)
{
    const double V = L * L * L;
    const double tp = 2.0 * M_PI / L;
    int side = 2 * mmax + 1;
    int K = side * side * side - 1;
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)K);
    int t = 0;
    for (int a = -mmax; a <= mmax; ++a)
        for (int b = -mmax; b <= mmax; ++b)
            for (int d = -mmax; d <= mmax; ++d) {
                if (a == 0 && b == 0 && d == 0) continue;
                m[3 * t] = a; m[3 * t + 1] = b; m[3 * t + 2] = d;
                ++t;
            }
    double *rre = (double *)calloc((size_t)K, sizeof(double));
    double *rim = (double *)calloc((size_t)K, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int l = 0; l < K; ++l) {
        double kx = tp * m[3 * l], ky = tp * m[3 * l + 1], kz = tp * m[3 * l + 2];
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < N; ++j) {
            double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
            sr += q[j] * cos(th);
            si += q[j] * sin(th);
        }
        rre[l] = sr; rim[l] = si;
    }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double s2 = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int l = 0; l < K; ++l) {
            double kx = tp * m[3 * l], ky = tp * m[3 * l + 1], kz = tp * m[3 * l + 2];
            double k2 = kx * kx + ky * ky + kz * kz;
            double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
            double im_part = cos(th) * rim[l] - sin(th) * rre[l];
            double ek = exp(-k2 / (4.0 * alpha));
            double g = 4.0 * M_PI * q[i] / (V * k2);
            fx -= g * ek * kx * im_part;
            fy -= g * ek * ky * im_part;
            fz -= g * ek * kz * im_part;
            s2 += (4.0 * M_PI * q[i]) * (4.0 * M_PI * q[i]) * S / (V * V * k2) * ek * im_part * im_part;
        }
        double f2 = fx * fx + fy * fy + fz * fz;
        var[i] = lB * lB * (s2 - f2) / (double)P;
        if (F1) { F1[3 * i] = lB * fx; F1[3 * i + 1] = lB * fy; F1[3 * i + 2] = lB * fz; }
    }
    free(m); free(rre); free(rim);
}

/* ------------------------------------------------------------------------- */
/* One Langevin step (Sec. 3.3: m dv = (F - gamma v) dt + sqrt(2 gamma kT)   */
/* dW) in the kick / exact Ornstein-Uhlenbeck / drift form:                  */
/*   v <- v + (dt/m) F;  v <- c1 v + c2 xi;  r <- wrap(r + dt v)             */
/* c1 = exp(-gamma dt / m), c2 = sqrt((1 - c1^2) kT / m).  The normals xi of  */
/* particle i come from Philox(key = seed, ctr = (i, 0, step_lo,             */
/* (stream << 8) | 2)) by Box-Muller on the uniforms u = (w+1) 2^-32 (words  */
/* 0 and 2) and w 2^-32 (words 1 and 3).                                     */
/* ------------------------------------------------------------------------- */
void orc_langevin_normals(int N, uint64_t seed, uint32_t stream, uint64_t step, double *xi)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < N; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, (uint32_t)step, (stream << 8) | 0x02u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        double u1 = ((double)w[0] + 1.0) / 4294967296.0;
        double u2 = (double)w[1] / 4294967296.0;
        double u3 = ((double)w[2] + 1.0) / 4294967296.0;
        double u4 = (double)w[3] / 4294967296.0;
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        xi[3 * i + 0] = r1 * cos(2.0 * M_PI * u2);
        xi[3 * i + 1] = r1 * sin(2.0 * M_PI * u2);
        xi[3 * i + 2] = r2 * cos(2.0 * M_PI * u4);
    }
}

void orc_langevin_step(int N, double *pos, double *vel, const double *F, double L,
                       double gamma, double kT, double dt, double mass,
                       uint64_t seed, uint32_t stream, uint64_t step)
{
    double *xi = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    orc_langevin_normals(N, seed, stream, step, xi);
    double c1 = exp(-gamma * dt / mass);
    double c2 = sqrt((1.0 - c1 * c1) * kT / mass);
    for (int i = 0; i < N; ++i) {
        for (int a = 0; a < 3; ++a) {
            double v = vel[3 * i + a] + (dt / mass) * F[3 * i + a];
            v = c1 * v + c2 * xi[3 * i + a];
            double r = pos[3 * i + a] + dt * v;
            r -= L * floor(r / L);
            vel[3 * i + a] = v;
            pos[3 * i + a] = r;
        }
    }
    free(xi);
}

/* ------------------------------------------------------------------------- */
/* Metropolis-Hastings sampling of the per-axis marginal P(m) as the paper    */
/* prints it (Sec. 3.1): the proposal m* = round(x*), x* ~ N(0, alpha L^2 /   */
/* (2 pi^2)), has the pmf                                                     */
/*   qbar(0) = erf(1/(2s)),                                                   */
/*   qbar(m) = (erf((|m|+1/2)/s) - erf((|m|-1/2)/s)) / 2,  s = sqrt(alpha) L/pi,*/
/* written here with erfc (same value, no cancellation in the tails).  The    */
/* chain is an independence sampler: from state m it accepts m* with          */
/* probability min(1, [P(m*)/qbar(m*)] / [P(m)/qbar(m)]) (the garbled         */
/* "accepted with probability q(m*|m)" read as the standard MH rule).  Three  */
/* independent chains give m_x, m_y, m_z; triples (0,0,0) are discarded; the  */
/* chain is consumed in order, P nonzero triples per step (the set K of       */
/* Algorithm 1).                                                              */
/*                                                                            */
/* Tables over |m| <= M (index j = m + M):                                    */
/*   Tq[j] = floor(2^32 * (sum_{i<=j} qbar_i) / (sum_all qbar)), Tq[2M] = 2^32 */
/*   rho[j] = exp(-pi^2 m^2 / (alpha L^2)) / qbar(m)   (ratios are what count) */
/* Iteration t of the chains: for axis c, w = Philox(key = seed,              */
/* ctr = (t_lo, t_hi, c, (stream << 8) | 6)); m* = inverse-CDF lookup of w0 in */
/* Tq; u = ((w2 << 32 | w3) >> 11) 2^-53; accept iff u * rho(m) < rho(m*).    */
/* ------------------------------------------------------------------------- */
void orc_mh_tables(double alpha, double L, int M, uint64_t *Tq, double *rho)
{
    const int n = 2 * M + 1;
    const double s = sqrt(alpha) * L / M_PI;
    const double a = (M_PI * M_PI) / (alpha * L * L);
    double *qb = (double *)malloc(sizeof(double) * (size_t)n);
    double Q = 0.0;
    for (int j = 0; j < n; ++j) {
        int m = j - M;
        int am = m < 0 ? -m : m;
        if (am == 0)
            qb[j] = erf(0.5 / s);
        else
            qb[j] = 0.5 * (erfc(((double)am - 0.5) / s) - erfc(((double)am + 0.5) / s));
        Q += qb[j];
    }
    double cum = 0.0;
    for (int j = 0; j < n; ++j) {
        cum += qb[j];
        if (j == n - 1) {
            Tq[j] = 4294967296ull;
        } else {
            double f = floor((cum / Q) * 4294967296.0);
            if (f > 4294967295.0) f = 4294967295.0;
            Tq[j] = (uint64_t)f;
        }
        long mm = (long)(j - M) * (long)(j - M);
        rho[j] = exp(-(a * (double)mm)) / qb[j];
    }
    free(qb);
}

/* Advance the three chains from state[3] / *pos (iterations done) until P
 * nonzero triples are emitted into m_out (P x 3).  Returns 0, or 1 if more
 * than 64 P + 1024 iterations were needed (then the rest is zero). */
int orc_mh_sample_k(double alpha, double L, uint64_t seed, uint32_t stream, int P,
                    int32_t *state, uint64_t *pos, int32_t *m_out)
{
    int M = orc_axis_M(alpha, L);
    int n = 2 * M + 1;
    uint64_t *Tq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    double *rho = (double *)malloc(sizeof(double) * (size_t)n);
    orc_mh_tables(alpha, L, M, Tq, rho);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t t = *pos;
    const uint64_t tmax = t + 64ull * (uint64_t)P + 1024ull;
    int emitted = 0, bad = 0;
    while (emitted < P) {
        if (t >= tmax) { bad = 1; break; }
        for (int c = 0; c < 3; ++c) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), (uint32_t)c, (stream << 8) | 0x06u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            int ms = orc_axis_lookup(Tq, M, w[0]);
            double u = (double)(((uint64_t)w[2] << 32 | (uint64_t)w[3]) >> 11) * 0x1.0p-53;
            volatile double lhs = u * rho[state[c] + M];     /* rounded product, no fma */
            if (lhs < rho[ms + M]) state[c] = ms;
        }
        ++t;
        if (state[0] != 0 || state[1] != 0 || state[2] != 0) {
            m_out[3 * emitted + 0] = state[0];
            m_out[3 * emitted + 1] = state[1];
            m_out[3 * emitted + 2] = state[2];
            ++emitted;
        }
    }
    for (int l = emitted; l < P; ++l) m_out[3 * l] = m_out[3 * l + 1] = m_out[3 * l + 2] = 0;
    *pos = t;
    free(Tq);
    free(rho);
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Leapfrog with the Andersen thermostat, the loop step of Algorithm 1 as    */
/* printed (Sec. 3.1, steps (2) and (3)):                                    */
/*   v^{n+1/2} = v^{n-1/2} + (dt/m) F^n;  r^{n+1} = wrap(r^n + dt v^{n+1/2}); */
/*   then, with probability nu dt, v^{n+1/2} <- N(0, kT/m) per component.    */
/* (The first call, from v^0, is the Euler start the paper mentions.)        */
/* Particle i at step n: collision iff w0 < floor(nu dt 2^32) with           */
/* w = Philox(key = seed, ctr = (i, 0, step_lo, (stream << 8) | 7)); the new  */
/* velocity's normals come from ctr = (i, 1, step_lo, (stream << 8) | 7) by   */
/* Box-Muller as in orc_langevin_normals.                                    */
/* ------------------------------------------------------------------------- */
void orc_andersen_step(int N, double *pos, double *vel, const double *F, double L,
                       double nu, double kT, double dt, double mass,
                       uint64_t seed, uint32_t stream, uint64_t step, int *collided)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double pc = nu * dt;
    double thr = floor(pc * 4294967296.0);
    if (thr > 4294967296.0) thr = 4294967296.0;
    double sd = sqrt(kT / mass);
    for (int i = 0; i < N; ++i) {
        for (int a = 0; a < 3; ++a) {
            double v = vel[3 * i + a] + (dt / mass) * F[3 * i + a];
            double r = pos[3 * i + a] + dt * v;
            r -= L * floor(r / L);
            vel[3 * i + a] = v;
            pos[3 * i + a] = r;
        }
        uint32_t c0[4] = {(uint32_t)i, 0u, (uint32_t)step, (stream << 8) | 0x07u};
        uint32_t w[4];
        orc_philox4x32_10(c0, key, w);
        int hit = (double)w[0] < thr;
        if (collided) collided[i] = hit;
        if (!hit) continue;
        uint32_t c1[4] = {(uint32_t)i, 1u, (uint32_t)step, (stream << 8) | 0x07u};
        orc_philox4x32_10(c1, key, w);
        double u1 = ((double)w[0] + 1.0) / 4294967296.0;
        double u2 = (double)w[1] / 4294967296.0;
        double u3 = ((double)w[2] + 1.0) / 4294967296.0;
        double u4 = (double)w[3] / 4294967296.0;
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        vel[3 * i + 0] = sd * r1 * cos(2.0 * M_PI * u2);
        vel[3 * i + 1] = sd * r1 * sin(2.0 * M_PI * u2);
        vel[3 * i + 2] = sd * r2 * cos(2.0 * M_PI * u4);
    }
}

/* ------------------------------------------------------------------------- */
/* True (non-random) energy and virial for the pressure (the paper computes  */
/* observables "without random batch").  Full Ewald with the cube            */
/* 0 < |m|_inf <= mmax, real space under r_c, shifted LJ under lj_rcut.      */
/* Virial W such that P = (2 E_kin + W) / (3 V), W = -dE/dlambda at lambda = */
/* 1 under r -> lambda r, L -> lambda L (alpha fixed):                       */
/*   real space  sum_{i<j} lB q_i q_j [erfc(sqrt(a) r)/r + 2 sqrt(a/pi) e^{-a r^2}] */
/*   Fourier     sum_k A_k |rho_k|^2 (1 - k^2 / (2 alpha)),                   */
/*               A_k = (2 pi lB / V) e^{-k^2/(4 alpha)} / k^2                 */
/*   background  3 E_bg,  E_bg = -lB pi (sum q)^2 / (2 V alpha); self: 0      */
/*   LJ          sum_{i<j} 24 eps (2 (s/r)^12 - (s/r)^6)                      */
/* out[0..3] = E_fourier (incl. self and background), E_real, E_lj, E_bg;    */
/* out[4..7] = W_fourier (reciprocal sum only), W_real, W_lj, W_bg.          */
/* ------------------------------------------------------------------------- */
void orc_true_energy_virial(int N, const double *pos, const double *q, double L, double alpha,
                            double r_c, double lB, double lj_eps, double lj_sigma,
                            double lj_rcut, int mmax, double *out)
{
    const double V = L * L * L, tp = 2.0 * M_PI / L;
    double sq = 0.0, sq2 = 0.0;
    for (int i = 0; i < N; ++i) { sq += q[i]; sq2 += q[i] * q[i]; }
    double ef = 0.0, wf = 0.0;
    #pragma omp parallel for schedule(dynamic) reduction(+ : ef, wf) collapse(2)
    for (int a = -mmax; a <= mmax; ++a)
        for (int b = -mmax; b <= mmax; ++b)
            for (int d = -mmax; d <= mmax; ++d) {
                if (a == 0 && b == 0 && d == 0) continue;
                double kx = tp * a, ky = tp * b, kz = tp * d;
                double k2 = kx * kx + ky * ky + kz * kz;
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < N; ++j) {
                    double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
                    sr += q[j] * cos(th);
                    si += q[j] * sin(th);
                }
                double A = 2.0 * M_PI * lB / V * exp(-k2 / (4.0 * alpha)) / k2;
                double e = A * (sr * sr + si * si);
                ef += e;
                wf += e * (1.0 - k2 / (2.0 * alpha));
            }
    const double ebg = -lB * M_PI * sq * sq / (2.0 * V * alpha);
    const double eself = -lB * sqrt(alpha / M_PI) * sq2;
    const double sa = sqrt(alpha), tsa = 2.0 * sqrt(alpha / M_PI);
    double vshift = 0.0;
    if (lj_eps != 0.0) {
        double s6 = pow(lj_sigma / lj_rcut, 6.0);
        vshift = -4.0 * lj_eps * (s6 * s6 - s6);
    }
    double er = 0.0, wr = 0.0, el = 0.0, wl = 0.0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : er, wr, el, wl)
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                double x = pos[3 * j + c] - pos[3 * i + c];
                x -= L * nearbyint(x / L);
                r2 += x * x;
            }
            double r = sqrt(r2);
            if (r < r_c) {
                double qq = lB * q[i] * q[j];
                er += qq * erfc(sa * r) / r;
                wr += qq * (erfc(sa * r) / r + tsa * exp(-alpha * r2));
            }
            if (lj_eps != 0.0 && r < lj_rcut) {
                double s2 = lj_sigma * lj_sigma / r2, s6 = s2 * s2 * s2;
                el += 4.0 * lj_eps * (s6 * s6 - s6) + vshift;
                wl += 24.0 * lj_eps * (2.0 * s6 * s6 - s6);
            }
        }
    out[0] = ef + eself + ebg;
    out[1] = er;
    out[2] = el;
    out[3] = ebg;
    out[4] = wf;
    out[5] = wr;
    out[6] = wl;
    out[7] = 3.0 * ebg;
}

/* ------------------------------------------------------------------------- */
/* Nose-Hoover thermostat (Sec. 3.3: dr/dt = p/m, dp/dt = F - xi p,           */
/* dxi/dt = (sum |p|^2/m - 3 N kT) / Q), discretised as a leapfrog in which  */
/* xi advances from the kinetic sum of the previous step's half-step         */
/* velocities and the friction enters symmetrically:                         */
/*   xi <- xi + (dt/Q) (K2 - 3 N kT)          (skipped on the first step)    */
/*   v  <- [v (1 - xi dt/2) + (dt/m) F] / (1 + xi dt/2);  r <- wrap(r + dt v) */
/*   K2 <- sum_i m |v_i|^2                                                    */
/* with Q = 3 N kT tau^2.  state[0] = xi, state[1] = K2, state[2] = 1 until  */
/* the first step has run (then 0).                                          */
/* ------------------------------------------------------------------------- */
void orc_nose_hoover_step(int N, double *pos, double *vel, const double *F, double L,
                          double tau, double kT, double dt, double mass, double *state)
{
    const double Q = 3.0 * (double)N * kT * tau * tau;
    if (state[2] == 0.0)
        state[0] += dt / Q * (state[1] - 3.0 * (double)N * kT);
    state[2] = 0.0;
    const double xi = state[0];
    const double a = 1.0 - 0.5 * xi * dt, b = 1.0 / (1.0 + 0.5 * xi * dt);
    double k2 = 0.0;
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < 3; ++c) {
            double v = (vel[3 * i + c] * a + (dt / mass) * F[3 * i + c]) * b;
            double r = pos[3 * i + c] + dt * v;
            r -= L * floor(r / L);
            vel[3 * i + c] = v;
            pos[3 * i + c] = r;
            k2 += mass * v * v;
        }
    }
    state[1] = k2;
}

/* ------------------------------------------------------------------------- */
/* Thread count of the OpenMP loops (for timing the oracle on one core and on */
/* all cores).  Each thread owns whole rows of every outer loop, so results   */
/* do not depend on this setting.  n <= 0 restores all available processors. */
/* ------------------------------------------------------------------------- */
#include <omp.h>
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }
int orc_get_threads(void) { return omp_get_max_threads(); }
