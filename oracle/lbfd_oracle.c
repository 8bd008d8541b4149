/*
 * ORACLE for the fluctuating lattice-Boltzmann diffusion step
 * (Wagner & Strand, "A Fluctuating Lattice Boltzmann Method for the
 * Diffusion Equation", arXiv:1606.07801).
 *
 * This file is TEST INFRASTRUCTURE.  It is a plain, slow, FP64 restatement
 * of the method, written to be checked against the paper by eye.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  The CUDA library shares no code, header, table or constant
 * generator with it.
 *
 * Order of operations follows the paper:
 *   - lattice velocities v_i and weights w_i with f^0_i = rho w_i
 *     (Sec. II, eqs. f0_0-f0_2, f0def; D2Q5 weights w_0 = 1-2 theta,
 *     w_1..4 = theta/2);
 *   - moment basis m_i^a by Gram-Schmidt under <a,b> = sum_i a_i w_i b_i,
 *     back-transform n_i^a = m_i^a w_i (Sec. II, the moment-matrix passage);
 *   - collision in moment space: M^a = sum_i m_i^a f_i,
 *     M^{a,0} = rho delta^{a0}, Lambda^{ab} = delta^{ab}/tau^a (eq. coll),
 *     noise xi^a with variance rho (2 tau^a - 1)/(tau^a)^2 for a >= 1
 *     (eq. xiglobal with rho^eq, eq. xilocal with the local rho, the local
 *     density clamped at zero as in Sec. IV "Simulation results");
 *   - back-transform f*_i = sum_a n_i^a M^{a*}, then streaming
 *     f_i(x + v_i, t+1) = f*_i(x) (eq. LB), periodic.
 *
 * The paper does not fix a random-number generator.  The noise here is
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3") keyed by (seed, lattice id, step, site,
 * call), turned into unit normals by the Box-Muller transform (Box &
 * Muller 1958), or into unit-variance uniforms on (-sqrt3, sqrt3) for the
 * flat distribution the paper itself uses (Sec. IV).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_D1Q3 0
#define ORC_D2Q9 1
#define ORC_D3Q19 2
#define ORC_D2Q5 3

#define ORC_NOISE_LOCAL 0
#define ORC_NOISE_GLOBAL 1
#define ORC_NOISE_OFF 2

#define ORC_GAUSSIAN 0
#define ORC_UNIFORM 1

#define ORC_QMAX 19

/* pi to double precision */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Lattices (Sec. II: f^0 = rho w_i with sum w = 1, sum w v = 0,       */
/* sum w v v = theta delta).  D2Q5 is the paper's own lattice; D1Q3,   */
/* D2Q9 and D3Q19 are the one/two/three-dimensional counterparts the   */
/* paper calls "near identical", all with theta = 1/3.                 */
/* ------------------------------------------------------------------ */

/* Fills D, Q, v[Q][3] and w[Q].  Returns 0, or -1 for an unknown lattice. */
int orc_lattice(int lat, double theta, int *D, int *Q, int *v, double *w)
{
    int i;
    for (i = 0; i < ORC_QMAX * 3; i++) v[i] = 0;
    if (lat == ORC_D1Q3) {
        static const int vx[3] = {0, 1, -1};
        *D = 1; *Q = 3;
        for (i = 0; i < 3; i++) v[3 * i] = vx[i];
        w[0] = 2.0 / 3.0; w[1] = 1.0 / 6.0; w[2] = 1.0 / 6.0;
        return 0;
    }
    if (lat == ORC_D2Q9) {
        static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                    {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
        *D = 2; *Q = 9;
        for (i = 0; i < 9; i++) { v[3 * i] = c[i][0]; v[3 * i + 1] = c[i][1]; }
        w[0] = 4.0 / 9.0;
        for (i = 1; i <= 4; i++) w[i] = 1.0 / 9.0;
        for (i = 5; i <= 8; i++) w[i] = 1.0 / 36.0;
        return 0;
    }
    if (lat == ORC_D3Q19) {
        static const int c[19][3] = {
            {0, 0, 0},
            {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
            {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
            {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
            {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        *D = 3; *Q = 19;
        for (i = 0; i < 19; i++) {
            v[3 * i] = c[i][0]; v[3 * i + 1] = c[i][1]; v[3 * i + 2] = c[i][2];
        }
        w[0] = 1.0 / 3.0;
        for (i = 1; i <= 6; i++) w[i] = 1.0 / 18.0;
        for (i = 7; i <= 18; i++) w[i] = 1.0 / 36.0;
        return 0;
    }
    if (lat == ORC_D2Q5) {
        /* velocity order and weights as printed in Sec. II */
        static const int c[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}};
        *D = 2; *Q = 5;
        for (i = 0; i < 5; i++) { v[3 * i] = c[i][0]; v[3 * i + 1] = c[i][1]; }
        w[0] = 1.0 - 2.0 * theta;
        for (i = 1; i <= 4; i++) w[i] = theta / 2.0;
        return 0;
    }
    return -1;
}

/* Seed vector a of the Gram-Schmidt procedure, evaluated at velocity v.
 * D2Q5: the paper's list 1, v_x, v_y, v_x^2 - v_y^2, v_x^2 + v_y^2.
 * D1Q3: 1, v, v^2.
 * D2Q9: v_x^p v_y^q with (p, q) in {0,1,2}^2, p-major.
 * D3Q19: v_x^p v_y^q v_z^r, p, q, r in {0,1,2}, at most two non-zero,
 *        ordered by total degree, then (p, q, r) descending. */
static double ipow(int x, int p)
{
    double r = 1.0;
    while (p-- > 0) r *= (double)x;
    return r;
}

static const int d3q19_mono[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
    {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 0, 2}, {0, 2, 1}, {0, 1, 2},
    {2, 2, 0}, {2, 0, 2}, {0, 2, 2}};

static double seed_vector(int lat, int a, const int *vi)
{
    int x = vi[0], y = vi[1], z = vi[2];
    switch (lat) {
    case ORC_D1Q3:
        return ipow(x, a);
    case ORC_D2Q9:
        return ipow(x, a / 3) * ipow(y, a % 3);
    case ORC_D3Q19:
        return ipow(x, d3q19_mono[a][0]) * ipow(y, d3q19_mono[a][1]) *
               ipow(z, d3q19_mono[a][2]);
    case ORC_D2Q5:
        switch (a) {
        case 0: return 1.0;
        case 1: return x;
        case 2: return y;
        case 3: return (double)(x * x - y * y);
        default: return (double)(x * x + y * y);
        }
    }
    return 0.0;
}

/* Moment basis m[a*Q + i] = m_i^a: Gram-Schmidt of the seed vectors under
 * the weighted scalar product sum_i m_i^a w_i m_i^b = delta^{ab}
 * (Sec. II, moment-matrix passage).  Returns Q, or -1 on a bad lattice or a
 * linearly dependent seed list. */
int orc_basis(int lat, double theta, double *m)
{
    int D, Q, v[ORC_QMAX * 3];
    double w[ORC_QMAX];
    int a, b, i;
    if (orc_lattice(lat, theta, &D, &Q, v, w) != 0) return -1;
    for (a = 0; a < Q; a++) {
        double u[ORC_QMAX], norm2 = 0.0;
        for (i = 0; i < Q; i++) u[i] = seed_vector(lat, a, &v[3 * i]);
        /* subtract the projections on the vectors already orthonormalised */
        for (b = 0; b < a; b++) {
            double proj = 0.0;
            for (i = 0; i < Q; i++) proj += u[i] * w[i] * m[b * Q + i];
            for (i = 0; i < Q; i++) u[i] -= proj * m[b * Q + i];
        }
        for (i = 0; i < Q; i++) norm2 += u[i] * w[i] * u[i];
        if (!(norm2 > 1e-12)) return -1;
        for (i = 0; i < Q; i++) m[a * Q + i] = u[i] / sqrt(norm2);
    }
    return Q;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).  Multipliers and Weyl key      */
/* increments are the published ones.                                  */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int r;
    for (r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1): the top 24 bits of a word, centred in their cell.
 * Every value is an odd multiple of 2^-25, exact in FP64. */
static double word_to_unit(uint32_t r)
{
    return ((double)(r >> 8) + 0.5) * (1.0 / 16777216.0);
}

/* Unit-variance noise variates z^1..z^nmom for one site and one step.
 * Philox call j has counter (site low word, lattice id, step low word,
 * step high word * 8 + j) and key (seed low word, seed high word); its four
 * outputs feed moments 4j+1 .. 4j+4.  Gaussian: Box-Muller on the pairs
 * (r0, r1) and (r2, r3).  Uniform: sqrt(3) (2u - 1) per word. */
void orc_site_noise(uint64_t seed, uint32_t lattice_id, uint64_t site,
                    uint64_t t, int nmom, int dist, double *z)
{
    int ncall = (nmom + 3) / 4, j, k;
    uint32_t key[2];
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    for (j = 0; j < ncall; j++) {
        uint32_t ctr[4], r[4];
        double zz[4], u[4];
        ctr[0] = (uint32_t)site;
        ctr[1] = lattice_id;
        ctr[2] = (uint32_t)t;
        ctr[3] = ((uint32_t)(t >> 32) << 3) | (uint32_t)j;
        orc_philox4x32_10(ctr, key, r);
        for (k = 0; k < 4; k++) u[k] = word_to_unit(r[k]);
        if (dist == ORC_GAUSSIAN) {
            double rad0 = sqrt(-2.0 * log(u[0]));
            double rad1 = sqrt(-2.0 * log(u[2]));
            zz[0] = rad0 * cos(2.0 * ORC_PI * u[1]);
            zz[1] = rad0 * sin(2.0 * ORC_PI * u[1]);
            zz[2] = rad1 * cos(2.0 * ORC_PI * u[3]);
            zz[3] = rad1 * sin(2.0 * ORC_PI * u[3]);
        } else {
            for (k = 0; k < 4; k++) zz[k] = sqrt(3.0) * (2.0 * u[k] - 1.0);
        }
        for (k = 0; k < 4; k++)
            if (4 * j + k < nmom) z[4 * j + k] = zz[k];
    }
}

/* ------------------------------------------------------------------ */
/* Collision of one site (eq. collision in moment space).              */
/* ------------------------------------------------------------------ */

/* Post-collision populations fout[Q] of one site from fin[Q], given the
 * unit variates z[0..Q-2] for moments a = 1..Q-1 and relaxation times
 * tau[0..Q-1] (tau[0] is irrelevant: the density is conserved).
 *   rho       = sum_i f_i
 *   M^a       = sum_i m_i^a f_i
 *   M^{a,0}   = rho delta^{a0}
 *   M^{a*}    = M^a + (M^{a,0} - M^a)/tau^a + xi^a,   xi^0 = 0
 *   xi^a      = sigma_a z^a,  sigma_a^2 = rho_n (2 tau^a - 1)/(tau^a)^2
 *   rho_n     = max(rho, 0) (local), rho_eq (global), none (off)
 *   f*_i      = sum_a n_i^a M^{a*},   n_i^a = m_i^a w_i
 * Returns 0, or -1 on a bad lattice. */
static void collide_site(int Q, const double *m, const double *w,
                         const double *tau, int noise_mode, double rho_eq,
                         const double *fin, const double *z, double *fout)
{
    double M[ORC_QMAX], rho = 0.0, rho_n;
    int a, i;
    for (i = 0; i < Q; i++) rho += fin[i];
    for (a = 0; a < Q; a++) {
        M[a] = 0.0;
        for (i = 0; i < Q; i++) M[a] += m[a * Q + i] * fin[i];
    }
    if (noise_mode == ORC_NOISE_LOCAL)
        rho_n = rho > 0.0 ? rho : 0.0;
    else if (noise_mode == ORC_NOISE_GLOBAL)
        rho_n = rho_eq;
    else
        rho_n = 0.0;
    for (a = 0; a < Q; a++) {
        double Meq = (a == 0) ? rho : 0.0;
        double xi = 0.0;
        if (a > 0 && noise_mode != ORC_NOISE_OFF) {
            double sigma = sqrt(rho_n * (2.0 * tau[a] - 1.0) / (tau[a] * tau[a]));
            xi = sigma * z[a - 1];
        }
        M[a] = M[a] + (Meq - M[a]) / tau[a] + xi;
    }
    for (i = 0; i < Q; i++) {
        fout[i] = 0.0;
        for (a = 0; a < Q; a++) fout[i] += m[a * Q + i] * w[i] * M[a];
    }
}

int orc_collide(int lat, double theta, const double *tau, int noise_mode,
                double rho_eq, const double *fin, const double *z, double *fout)
{
    int D, Q, v[ORC_QMAX * 3];
    double w[ORC_QMAX], m[ORC_QMAX * ORC_QMAX];
    if (orc_lattice(lat, theta, &D, &Q, v, w) != 0) return -1;
    if (orc_basis(lat, theta, m) != Q) return -1;
    collide_site(Q, m, w, tau, noise_mode, rho_eq, fin, z, fout);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Whole-lattice evolution (eq. LB): collide every site, then push      */
/* f*_i(x) to x + v_i with periodic wrap.                               */
/* ------------------------------------------------------------------ */

static int64_t wrap(int64_t c, int64_t L)
{
    c %= L;
    return c < 0 ? c + L : c;
}

/* Evolves f (layout f[i*N + site], site = x + Lx (y + Ly z)) in place by
 * nsteps steps, starting at step counter t0.  dims holds Lx, Ly, Lz (unused
 * trailing dimensions are 1).  Returns 0, or -1 on bad arguments / memory. */
int orc_run(int lat, double theta, const int64_t *dims, const double *tau,
            int noise_mode, int dist, double rho_eq, uint64_t seed,
            uint32_t lattice_id, uint64_t t0, int64_t nsteps, double *f)
{
    int D, Q, v[ORC_QMAX * 3];
    double w[ORC_QMAX], m[ORC_QMAX * ORC_QMAX];
    int64_t Lx = dims[0], Ly = dims[1], Lz = dims[2], N, step;
    double *g;
    if (orc_lattice(lat, theta, &D, &Q, v, w) != 0) return -1;
    if (orc_basis(lat, theta, m) != Q) return -1;
    if (Lx < 1 || Ly < 1 || Lz < 1 || nsteps < 0) return -1;
    N = Lx * Ly * Lz;
    g = (double *)malloc(sizeof(double) * (size_t)Q * (size_t)N);
    if (!g) return -1;
    for (step = 0; step < nsteps; step++) {
        uint64_t t = t0 + (uint64_t)step;
        int64_t s;
#pragma omp parallel for schedule(static)
        for (s = 0; s < N; s++) {
            double fin[ORC_QMAX], fout[ORC_QMAX], z[ORC_QMAX];
            int64_t x = s % Lx, y = (s / Lx) % Ly, zc = s / (Lx * Ly);
            int i;
            for (i = 0; i < Q; i++) fin[i] = f[(int64_t)i * N + s];
            for (i = 0; i < Q - 1; i++) z[i] = 0.0;
            if (noise_mode != ORC_NOISE_OFF)
                orc_site_noise(seed, lattice_id, (uint64_t)s, t, Q - 1, dist, z);
            collide_site(Q, m, w, tau, noise_mode, rho_eq, fin, z, fout);
            for (i = 0; i < Q; i++) {
                int64_t xd = wrap(x + v[3 * i], Lx);
                int64_t yd = wrap(y + v[3 * i + 1], Ly);
                int64_t zd = wrap(zc + v[3 * i + 2], Lz);
                g[(int64_t)i * N + xd + Lx * (yd + Ly * zd)] = fout[i];
            }
        }
        memcpy(f, g, sizeof(double) * (size_t)Q * (size_t)N);
    }
    free(g);
    return 0;
}

/* Local equilibrium start f_i(x, 0) = w_i rho(x, 0) (eq. f0def). */
int orc_init_equilibrium(int lat, double theta, int64_t N, const double *rho,
                         double *f)
{
    int D, Q, v[ORC_QMAX * 3], i;
    double w[ORC_QMAX];
    int64_t s;
    if (orc_lattice(lat, theta, &D, &Q, v, w) != 0) return -1;
    for (i = 0; i < Q; i++)
        for (s = 0; s < N; s++) f[(int64_t)i * N + s] = w[i] * rho[s];
    return 0;
}
