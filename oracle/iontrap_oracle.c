/*
 * iontrap_oracle.c -- plain FP64 CPU oracle of the trapped-ion timestep.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of
 * the benchmark call it; the product library never does, and it shares no code,
 * header or constant with the CUDA path.
 *
 * What it computes (all FP64, SI units, slow and direct on purpose):
 *
 *   acceleration of ion i at positions x, time t, drag velocity u, noise counter n:
 *     a_i = (k_e Q_i / M_i) sum_{j != i} Q_j (x_i - x_j) / |x_i - x_j|^3     Eq. 4 (force
 *                                              of the pair term), direct sum, Sec. 6
 *                                              "Interactions" (brute force, no cutoff)
 *         + trap_i(x_i, t)                     Eq. 1 in the Mathieu a/q form of Eq. 3
 *         - gamma_i u_i + sigma_i xi_i(n)      Langevin bath, Sec. 3 "Cooling the
 *                                              motion of ions" (gamma = 1/dampingTime;
 *                                              a bath may act on a group of ions only,
 *                                              so gamma_i and T_i are per ion)
 *         - |g_i| (g^_i . u_i) g^_i            laser cooling laserCool(species, g),
 *                                              Sec. 3 "Cooling the motion of ions": a
 *                                              viscous force along the beam direction
 *                                              g^ = g/|g| at rate |g| (1/s), no kicks
 *
 *   trap_i for an ion whose charge/mass is rho times that of the reference species:
 *     x: -(Omega^2/4)(rho a - 2 rho q cos Omega t) x + (rho omega_z^2 / 2) x
 *     y: -(Omega^2/4)(rho a + 2 rho q cos Omega t) y + (rho omega_z^2 / 2) y
 *     z: -rho omega_z^2 z
 *   (q_x = -q_y = q, Eq. 3; a and q scale with Q/M, Eq. 3; the static axial field
 *    confines along z and defocuses radially by half its strength, Eq. 1 and 3.)
 *
 *   sigma_i = sqrt(2 gamma_i k_B T_i / (M_i dt)); xi = three standard normals drawn by
 *   Box-Muller from Philox-4x64-10 (Salmon et al., SC'11) with key (seed, 0) and
 *   counter (n, i, 0, 0), on the uniforms (top 23 bits + 1/2) 2^-23.
 *
 *   one step, velocity Verlet ("nve", Sec. 6 "Integration"), kick-drift-kick:
 *     v_half = v_n + dt/2 a_n
 *     x_{n+1} = x_n + dt v_half
 *     a_{n+1} = accel(x_{n+1}, t = (n+1) dt, u = v_half, counter n+1)
 *     v_{n+1} = v_half + dt/2 a_{n+1}
 *   and a_0 = accel(x_0, t = n0 dt, u = v_0, counter n0) before the first step.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction, so
 * x86 and Arm hosts give the same bits).  OpenMP only splits the loop over ions i;
 * each ion's sum over j runs in plain j order.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 */
static const double ORC_E = 1.602176634e-19;      /* C (exact) */
static const double ORC_KB = 1.380649e-23;        /* J/K (exact) */
static const double ORC_EPS0 = 8.8541878128e-12;  /* F/m */
static const double ORC_AMU = 1.66053906660e-27;  /* kg */
static const double ORC_PI = 3.14159265358979323846;

#define ORC_RF_OFF 1u
#define ORC_COULOMB_OFF 2u
#define ORC_TRAP_OFF 4u
#define ORC_PSEUDO 16u   /* the trap is its Eq. 2 pseudopotential: static springs */

typedef struct {
    double Omega;    /* RF angular frequency, rad/s */
    double a;        /* Mathieu a of the reference species (x and y) */
    double q;        /* Mathieu q = q_x = -q_y of the reference species */
    double omega_z;  /* axial angular frequency of the reference species, rad/s */
    double gamma;    /* Langevin damping rate, 1/s */
    double T_bath;   /* bath temperature, K */
    double dt;       /* time step, s */
    uint64_t seed;   /* noise key */
    uint32_t flags;  /* ORC_* bits */
    uint32_t pad_;
    double qm_ref;   /* charge/mass of the reference species, C/kg */
} oracle_params;

double oracle_const(int which)
{
    switch (which) {
    case 0: return ORC_E;
    case 1: return ORC_KB;
    case 2: return ORC_EPS0;
    case 3: return ORC_AMU;
    default: return 1.0 / (4.0 * ORC_PI * ORC_EPS0);
    }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- Philox-4x64-10 */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
 * ten rounds of two 64x64->128 multiplications and a key schedule bumped by the
 * Weyl constants (golden ratio and sqrt(3)-1 in 0.64 fixed point). */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        if (round > 0) { k0 += W0; k1 += W1; }
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (seed, counter, ion id): the top 23 bits of each of the
 * four 64-bit Philox words give u_k = (m_k + 1/2) 2^-23 in (0, 1) (exact in FP32 as
 * well as FP64); Box-Muller turns (u0, u1) into two normals and (u2, u3) into the
 * third. */
void oracle_normals(uint64_t seed, int64_t counter, int64_t id, double z[3])
{
    uint64_t ctr[4] = {(uint64_t)counter, (uint64_t)id, 0u, 0u};
    uint64_t key[2] = {seed, 0u};
    uint64_t r[4];
    double u[4];
    oracle_philox4x64_10(ctr, key, r);
    for (int k = 0; k < 4; ++k) u[k] = ((double)(r[k] >> 41) + 0.5) * 0x1p-23;
    double R1 = sqrt(-2.0 * log(u[0]));
    double R2 = sqrt(-2.0 * log(u[2]));
    z[0] = R1 * cos(2.0 * ORC_PI * u[1]);
    z[1] = R1 * sin(2.0 * ORC_PI * u[1]);
    z[2] = R2 * cos(2.0 * ORC_PI * u[3]);
}

void oracle_normals_many(uint64_t seed, int64_t counter, int64_t m, const int64_t *ids,
                         double *z /* [3][m] */)
{
    for (int64_t k = 0; k < m; ++k) {
        double t[3];
        oracle_normals(seed, counter, ids[k], t);
        z[k] = t[0];
        z[m + k] = t[1];
        z[2 * m + k] = t[2];
    }
}

/* ------------------------------------------------------------------ Coulomb term */
/* Coulomb acceleration of the ions listed in idx (all ions when idx == NULL):
 * acc[c*m + k] = k_e Q_i / M_i * sum_{j != i} Q_j (x_i - x_j)_c / r_ij^3, i = idx[k].
 * x is SoA [3][n]. */
void oracle_coulomb_accel(int64_t n, const double *x, const double *charge,
                          const double *mass, const int64_t *idx, int64_t m, double *acc)
{
    const double ke = 1.0 / (4.0 * ORC_PI * ORC_EPS0);
    const double *X = x, *Y = x + n, *Z = x + 2 * n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = X[i] - X[j];
            double dy = Y[i] - Y[j];
            double dz = Z[i] - Z[j];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double f = charge[j] / (r2 * r);
            sx += f * dx;
            sy += f * dy;
            sz += f * dz;
        }
        double c = ke * charge[i] / mass[i];
        acc[k] = c * sx;
        acc[m + k] = c * sy;
        acc[2 * m + k] = c * sz;
    }
}

/* ---------------------------------------------------------------------- trap term */
/* Spring constants (1/s^2) of the pseudopotential of the trap for an ion of
 * charge/mass qm (Eq. 2): omega_m^2 = (Omega^2/4)(a_m + q_m^2/2) along x and y, with
 * q_m = rho q and a_m = rho a - 2 rho omega_z^2 / Omega^2 (the species' own dc a plus the
 * axial field's radial defocusing, Eq. 3: a_x = -a_z/2), and rho omega_z^2 along z. */
void oracle_pseudo_springs(const oracle_params *p, double qm, double k[3])
{
    double rho = qm / p->qm_ref;
    double O2 = p->Omega * p->Omega;
    double wz2 = rho * p->omega_z * p->omega_z;
    double a_m = rho * p->a - 2.0 * wz2 / O2;
    double q_m = rho * p->q;
    double kr = O2 / 4.0 * (a_m + 0.5 * q_m * q_m);
    k[0] = kr;
    k[1] = kr;
    k[2] = wz2;
}

/* Linear Paul trap acceleration (Eq. 1 with the Mathieu parameters of Eq. 3), or its
 * pseudopotential (Eq. 2) when ORC_PSEUDO is set. */
void oracle_trap_accel(const oracle_params *p, double qm, const double r[3], double t,
                       double acc[3])
{
    if (p->flags & ORC_TRAP_OFF) {
        acc[0] = acc[1] = acc[2] = 0.0;
        return;
    }
    if (p->flags & ORC_PSEUDO) {
        double k[3];
        oracle_pseudo_springs(p, qm, k);
        for (int c = 0; c < 3; ++c) acc[c] = -k[c] * r[c];
        return;
    }
    double rho = qm / p->qm_ref;
    double cosv = (p->flags & ORC_RF_OFF) ? 0.0 : cos(p->Omega * t);
    double quarter_O2 = p->Omega * p->Omega / 4.0;
    double wz2 = rho * p->omega_z * p->omega_z;
    double kx = quarter_O2 * (rho * p->a - 2.0 * rho * p->q * cosv);
    double ky = quarter_O2 * (rho * p->a + 2.0 * rho * p->q * cosv);
    acc[0] = -kx * r[0] + 0.5 * wz2 * r[0];
    acc[1] = -ky * r[1] + 0.5 * wz2 * r[1];
    acc[2] = -wz2 * r[2];
}

/* ------------------------------------------------------------- full acceleration */
/* Per-ion cooling (any pointer may be NULL):
 *   gamma[n], T_bath[n]  Langevin rate (1/s) and bath temperature (K) of each ion's bath;
 *                        NULL: every ion in the bath of p (p->gamma, p->T_bath)
 *   laser[3][n]          laser-cooling vector g of each ion (1/s, SoA; zero vector = no
 *                        laser); NULL: no laser cooling
 * A bath restricted to a group (langevinBath(T, dampingTime, group)) is a group whose
 * ions carry that bath's (gamma, T) and the others (0, 0). */
/* springs[3][n] (may be NULL): static spring constants k of each ion (1/s^2, SoA),
 * acceleration -k_c x_c, replacing the trap of p (a pseudopotential trap given by its
 * frequencies, linearPseudoPT, Sec. 3 "Forces and fields"). */
void oracle_accel_ex(int64_t n, const double *x, const double *udrag, const double *charge,
                     const double *mass, const oracle_params *p, int64_t counter, double t,
                     const double *gamma, const double *T_bath, const double *laser,
                     const double *springs, double *acc)
{
    if (p->flags & ORC_COULOMB_OFF) {
        for (int64_t k = 0; k < 3 * n; ++k) acc[k] = 0.0;
    } else {
        oracle_coulomb_accel(n, x, charge, mass, NULL, n, acc);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double r[3] = {x[i], x[n + i], x[2 * n + i]};
        double u[3] = {udrag[i], udrag[n + i], udrag[2 * n + i]};
        double tr[3];
        if (springs)
            for (int c = 0; c < 3; ++c) tr[c] = -springs[c * n + i] * r[c];
        else
            oracle_trap_accel(p, charge[i] / mass[i], r, t, tr);
        double g_i = gamma ? gamma[i] : p->gamma;
        double T_i = gamma ? T_bath[i] : p->T_bath;
        double sigma = sqrt(2.0 * g_i * ORC_KB * T_i / (mass[i] * p->dt));
        double xi[3] = {0.0, 0.0, 0.0};
        if (sigma > 0.0) oracle_normals(p->seed, counter, i, xi);
        /* laser: -|g| (g^ . u) g^ with g^ = g / |g| */
        double las[3] = {0.0, 0.0, 0.0};
        if (laser) {
            double g[3] = {laser[i], laser[n + i], laser[2 * n + i]};
            double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            if (gn > 0.0) {
                double khat[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
                double proj = khat[0] * u[0] + khat[1] * u[1] + khat[2] * u[2];
                for (int c = 0; c < 3; ++c) las[c] = -gn * proj * khat[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            double lang = -g_i * u[c] + sigma * xi[c];
            acc[c * n + i] += tr[c] + lang + las[c];
        }
    }
}

void oracle_accel(int64_t n, const double *x, const double *udrag, const double *charge,
                  const double *mass, const oracle_params *p, int64_t counter, double t,
                  double *acc)
{
    oracle_accel_ex(n, x, udrag, charge, mass, p, counter, t, NULL, NULL, NULL, NULL, acc);
}

/* ------------------------------------------------------------ velocity Verlet run */
/* Advances (x, v, a) in place by nsteps from step index step0.  With init != 0 it
 * first evaluates a_0 at (x_0, t = step0 dt) with v_0 as the drag velocity. */
/* Changing the forces between two runs (interleaved evolve, Sec. 3 "Time evolution")
 * is a second call with the new parameters and init != 0: a_n is re-evaluated under the
 * new forces at (x_n, t = n dt), with v_n as the drag velocity and noise counter n. */
void oracle_run_ex(int64_t n, double *x, double *v, double *a, const double *charge,
                   const double *mass, const oracle_params *p, int64_t step0, int64_t nsteps,
                   int init, const double *gamma, const double *T_bath, const double *laser,
                   const double *springs, double *work /* 3n doubles of scratch */)
{
    const double dt = p->dt;
    if (init)
        oracle_accel_ex(n, x, v, charge, mass, p, step0, (double)step0 * dt, gamma, T_bath,
                        laser, springs, a);
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t step = step0 + s;
        double *vh = work;
        for (int64_t k = 0; k < 3 * n; ++k) {
            vh[k] = v[k] + 0.5 * dt * a[k];
            x[k] = x[k] + dt * vh[k];
        }
        oracle_accel_ex(n, x, vh, charge, mass, p, step + 1, (double)(step + 1) * dt, gamma,
                        T_bath, laser, springs, a);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] = vh[k] + 0.5 * dt * a[k];
    }
}

void oracle_run(int64_t n, double *x, double *v, double *a, const double *charge,
                const double *mass, const oracle_params *p, int64_t step0, int64_t nsteps,
                int init, double *work /* 3n doubles of scratch */)
{
    oracle_run_ex(n, x, v, a, charge, mass, p, step0, nsteps, init, NULL, NULL, NULL, NULL, work);
}

/* ------------------------------------------------------------------------ energy */
/* Total energy for a static trap (RF off, the pseudopotential of Eq. 2, or the static
 * springs[3][n] when given): kinetic + trap potential + Coulomb pair potential (Eq. 4,
 * each unordered pair once). */
double oracle_energy_ex(int64_t n, const double *x, const double *v, const double *charge,
                        const double *mass, const oracle_params *p, const double *springs)
{
    const double ke = 1.0 / (4.0 * ORC_PI * ORC_EPS0);
    double kin = 0.0, trap = 0.0, coul = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = 0.0;
        for (int c = 0; c < 3; ++c) v2 += v[c * n + i] * v[c * n + i];
        kin += 0.5 * mass[i] * v2;
        if (springs || (p->flags & ORC_PSEUDO)) {
            double k[3];
            if (springs)
                for (int c = 0; c < 3; ++c) k[c] = springs[c * n + i];
            else
                oracle_pseudo_springs(p, charge[i] / mass[i], k);
            for (int c = 0; c < 3; ++c) trap += 0.5 * mass[i] * k[c] * x[c * n + i] * x[c * n + i];
        } else if (!(p->flags & ORC_TRAP_OFF)) {
            double rho = (charge[i] / mass[i]) / p->qm_ref;
            double wz2 = rho * p->omega_z * p->omega_z;
            double kr = p->Omega * p->Omega / 4.0 * rho * p->a - 0.5 * wz2;
            double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
            trap += 0.5 * mass[i] * (kr * xi * xi + kr * yi * yi + wz2 * zi * zi);
        }
    }
    if (!(p->flags & ORC_COULOMB_OFF)) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                double dx = x[i] - x[j], dy = x[n + i] - x[n + j], dz = x[2 * n + i] - x[2 * n + j];
                coul += ke * charge[i] * charge[j] / sqrt(dx * dx + dy * dy + dz * dz);
            }
    }
    return kin + trap + coul;
}

double oracle_energy(int64_t n, const double *x, const double *v, const double *charge,
                     const double *mass, const oracle_params *p)
{
    return oracle_energy_ex(n, x, v, charge, mass, p, NULL);
}

/* ----------------------------------------------------------------------- Hessian */
/* Mass-weighted Hessian of the static potential (trap springs + Coulomb pair energy of
 * Eq. 4) at positions x: H[(3i+a)(3n) + 3j+b] = d^2 V / dx_ia dx_jb / sqrt(M_i M_j).
 * Its eigenvalues are the squared normal-mode frequencies (Sec. 5 "Normal modes of
 * motion").  Pair block (i != j), r = x_i - x_j:
 *   d^2 (k_e Q_i Q_j / |r|) / dx_ia dx_jb = k_e Q_i Q_j (delta_ab / r^3 - 3 r_a r_b / r^5)
 * and the diagonal block is minus the sum of the pair blocks of row i plus M_i k_a delta_ab
 * (the pair energy depends on x_i - x_j only).  springs[3][n] as for oracle_accel_ex, or
 * NULL for the pseudopotential of p (Eq. 2). */
void oracle_hessian(int64_t n, const double *x, const double *charge, const double *mass,
                    const oracle_params *p, const double *springs, double *H)
{
    const double ke = 1.0 / (4.0 * ORC_PI * ORC_EPS0);
    const int64_t m = 3 * n;
    for (int64_t k = 0; k < m * m; ++k) H[k] = 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double diag[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3], r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                r[c] = x[c * n + i] - x[c * n + j];
                r2 += r[c] * r[c];
            }
            double rr = sqrt(r2);
            double r3 = r2 * rr, r5 = r3 * r2;
            double kq = ke * charge[i] * charge[j];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double hab = kq * ((a == b ? 1.0 : 0.0) / r3 - 3.0 * r[a] * r[b] / r5);
                    H[(3 * i + a) * m + 3 * j + b] = hab / sqrt(mass[i] * mass[j]);
                    diag[a][b] -= hab;
                }
        }
        double k[3];
        if (springs)
            for (int c = 0; c < 3; ++c) k[c] = springs[c * n + i];
        else
            oracle_pseudo_springs(p, charge[i] / mass[i], k);
        for (int a = 0; a < 3; ++a) {
            diag[a][a] += mass[i] * k[a];
            for (int b = 0; b < 3; ++b) H[(3 * i + a) * m + 3 * i + b] = diag[a][b] / mass[i];
        }
    }
}
