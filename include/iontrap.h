/*
 * iontrap.h -- C ABI of libiontrap.so, a GB300 (sm_103a) library that advances N
 * trapped ions in a linear Paul trap with a Langevin bath, by velocity Verlet, with
 * the all-pairs Coulomb force summed on the GPU.
 *
 * The problem statement follows (py)LIon (arxiv 1907.10514):
 *   - species defined by charge (units of e) and mass (amu)   Sec. 3 "Adding ions"
 *   - ions placed at given coordinates, ids = index order      Sec. 3 "Adding ions"
 *   - linear Paul trap, full RF field, Mathieu a/q form         Eq. 1, Eq. 3, Sec. 3 "Forces and fields"
 *   - Langevin bath langevinBath(T, dampingTime[, group])       Sec. 3 "Cooling the motion of ions"
 *   - laser cooling laserCool(species, gamma)                    Sec. 3 "Cooling the motion of ions"
 *   - forces changed between evolve calls                        Sec. 3 "Time evolution"
 *   - all-pairs Coulomb interaction, no cutoff                  Eq. 4, Sec. 6 "Interactions"
 *   - evolve(N): N steps of the "nve" integrator                Sec. 3 "Time evolution", Sec. 6 "Integration"
 *   - positions and velocities read back in id order            Sec. 3 "Writing/reading data"
 *   - parameters change only between evolve calls              Sec. 3 "Time evolution", "Execution"
 *
 * One step (index n -> n+1), for every ion i with charge number z_i and mass M_i:
 *   v_half  = v_n + dt/2 a_n
 *   x_{n+1} = x_n + dt v_half
 *   a_{n+1} = (k_e e^2 z_i / M_i) sum_{j != i} z_j (x_i - x_j) / |x_i - x_j|^3
 *           + trap_i(x_{n+1}, t_{n+1}) - gamma_s v_half + sigma_i xi_i(n+1)
 *           - |g_s| (g^_s . v_half) g^_s
 *   v_{n+1} = v_half + dt/2 a_{n+1}
 * with, for an ion whose charge/mass is rho times that of species 0 (c = cos Omega t):
 *   trap_x = -(Omega^2/4) rho (a - 2 q c) x + (rho omega_z^2 / 2) x
 *   trap_y = -(Omega^2/4) rho (a + 2 q c) y + (rho omega_z^2 / 2) y
 *   trap_z = -rho omega_z^2 z
 *   sigma_i = sqrt(2 gamma_s k_B T_s / (M_i dt)),  xi = 3 normals from Philox-4x64-10
 *   (key (seed, 0), counter (n+1, i, 0, 0)) by Box-Muller on the uniforms
 *   (top 23 bits of each 64-bit word + 1/2) 2^-23.
 * where (gamma_s, T_s) is the Langevin bath and g_s the laser-cooling vector of ion i's
 * species s (g^ = g/|g|; by default every species is in the bath of iontrap_params and
 * none is laser-cooled, see iontrap_set_params).
 * a_{n0} is evaluated at create time from (x_{n0}, t = n0 dt) with v_{n0} as drag.
 *
 * Layout: every per-ion array is SoA, [3][n] doubles (x block, then y, then z), in
 * metres and metres per second, SI throughout.  Ion id = array index.
 *
 * Ownership: the caller owns every host array it passes; the library copies in at
 * create and copies out in iontrap_state / iontrap_forces.  A handle owns its device
 * memory, its CUDA graph and (if it created one) its stream; iontrap_destroy frees
 * them.  Handles are not thread-safe; distinct handles may be used from distinct
 * threads.
 *
 * Errors: every int-returning call returns an IONTRAP_* status.  A device-side
 * failure (non-finite state, expired bounded wait, CUDA error) is sticky: the handle
 * returns the same status from then on and must be destroyed.
 */
#ifndef IONTRAP_H
#define IONTRAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IONTRAP_OK 0
#define IONTRAP_EINVAL 1      /* bad argument: n < 1, unknown species, non-finite input, dt < 0, ... */
#define IONTRAP_ENOMEM 2      /* device allocation failed */
#define IONTRAP_EUNSTABLE 3   /* a species' single-ion motion is unbounded under the discrete map */
#define IONTRAP_ENONFINITE 4  /* a step produced a non-finite acceleration, velocity or position */
#define IONTRAP_ETIMEOUT 5    /* a bounded device-side wait expired */
#define IONTRAP_ECUDA 6       /* a CUDA runtime call failed */
#define IONTRAP_ETOOLARGE 7   /* n exceeds the fixed scratch of iontrap_forces_noalloc */

/* iontrap_params.flags */
#define IONTRAP_RF_OFF 1u            /* drop the RF (q) term: static trap */
#define IONTRAP_COULOMB_OFF 2u       /* non-interacting ions */
#define IONTRAP_TRAP_OFF 4u          /* free ions: no trap field at all */
#define IONTRAP_ALLOW_UNSTABLE 8u    /* skip the stability check at create */
#define IONTRAP_PSEUDO 16u           /* pseudopotential trap (Eq. 2): static springs per species,
                                        (Omega^2/4)(a_s + q_s^2/2) radially with a_s = rho a -
                                        2 rho omega_z^2/Omega^2, q_s = rho q, and rho omega_z^2
                                        axially; or the frequencies of
                                        iontrap_set_pseudo_frequencies */

/* iontrap_params.precision */
#define IONTRAP_PREC_FP32 0  /* FP32 pair forces with compensated accumulation; FP64 state,
                                Verlet update and RF phase */
#define IONTRAP_PREC_FP64 1  /* plain form: FP64 everywhere (comparison baseline) */

#define IONTRAP_MAX_SPECIES 16

typedef struct {
    double mass_amu;  /* mass in atomic mass units, > 0 */
    double charge_e;  /* charge in units of e */
} iontrap_species;

typedef struct {
    double Omega;      /* RF angular frequency, rad/s (> 0 unless RF and trap are off) */
    double a;          /* Mathieu a of species 0, applied to x and y (Eq. 3) */
    double q;          /* Mathieu q of species 0: q_x = q, q_y = -q (Eq. 3) */
    double omega_z;    /* axial angular secular frequency of species 0, rad/s */
    double gamma;      /* Langevin damping rate 1/dampingTime, 1/s (0 = no bath) */
    double T_bath;     /* bath temperature, K */
    double dt;         /* time step, s; 0 selects 2 pi / Omega / 20 */
    uint64_t seed;     /* key of the Langevin noise stream */
    uint32_t flags;    /* IONTRAP_* flag bits */
    int32_t precision; /* IONTRAP_PREC_FP32 or IONTRAP_PREC_FP64 */
} iontrap_params;

typedef struct iontrap iontrap_t;

/* Create a simulation of n ions on the current CUDA device.
 *   species[n_species]     species table (1 <= n_species <= IONTRAP_MAX_SPECIES);
 *                          species 0 is the reference of a, q, omega_z
 *   species_of_ion[n]      species index of each ion
 *   x0[3n], v0[3n]         initial positions / velocities, SoA; v0 may be NULL (zeros)
 *   step0                  index of the initial state: t0 = step0 dt, noise counter step0
 *   cuda_stream            cudaStream_t to run on, or NULL for a stream the handle owns
 * Copies the inputs to the device, evaluates a_{step0} and returns the handle in *out.
 * The handle's device buffers come from a per-device pool of CUDA's stream-ordered
 * allocator, allocated and later freed in order on the handle's stream (neither
 * synchronises the device); the pool keeps up to 4 GiB of freed memory for reuse.
 * EINVAL on bad arguments, EUNSTABLE if the trap cannot hold a species (unless
 * IONTRAP_ALLOW_UNSTABLE), ENOMEM / ECUDA on device failure.  Synchronous. */
int iontrap_create(const iontrap_species *species, int n_species,
                   const uint8_t *species_of_ion, const double *x0, const double *v0,
                   int64_t n, const iontrap_params *p, int64_t step0, void *cuda_stream,
                   iontrap_t **out);

/* Enqueue n_steps >= 0 velocity-Verlet steps (Sec. 3 "Time evolution", evolve(N)) on the
 * handle's stream.  Asynchronous: returns once the work is enqueued (as CUDA graphs of
 * 100 steps plus single launches).  Returns the handle's sticky status. */
int iontrap_step(iontrap_t *h, int64_t n_steps);

/* Cooling of one species (Sec. 3 "Cooling the motion of ions").  A Langevin bath
 * langevinBath(T, dampingTime, group) with the group one species: drag -gamma v and
 * Gaussian kicks of variance 2 gamma k_B T / (M dt) per component and step.  Laser cooling
 * laserCool(species, g): a viscous force along the beam, acceleration -|g| (g^.v) g^ with
 * g^ = g/|g|, no kicks (the paper writes the force as -M (g.v) g; its examples give g as a
 * rate in 1/s times a direction, which is the reading taken here).  v is the half-step
 * velocity, as for the bath.  To give a group of ions of one kind a bath of its own,
 * declare it as a separate species with the same mass and charge. */
typedef struct {
    double gamma;     /* bath rate 1/dampingTime, 1/s (0 = no bath) */
    double T_bath;    /* bath temperature, K */
    double laser[3];  /* laser-cooling vector g, 1/s (zero vector = no laser cooling) */
} iontrap_cooling;

/* Change the forces between evolve calls (Sec. 3 "Time evolution": interleaving evolve
 * with commands that add or remove forces and fields; Sec. 4 Example 2 removes a bath and
 * laser-cools one species).  From the current state n on, the trap is that of p (Omega,
 * a, q, omega_z, IONTRAP_RF_OFF / IONTRAP_TRAP_OFF) and species s has the bath and laser of
 * cooling[s] (cooling[n_species], or NULL: every species in the bath (p->gamma, p->T_bath),
 * no laser).  The state keeps x_n and v_n; a_n is evaluated again under the new forces
 * exactly as iontrap_create evaluates it (at t = n dt, drag on v_n, noise counter n), so the
 * handle continues bit for bit like a handle created from (x_n, v_n) at step0 = n with the
 * new forces.  dt, seed, precision and IONTRAP_COULOMB_OFF cannot change (EINVAL).
 * EINVAL on non-finite or negative bath values, EUNSTABLE for a trap that cannot hold a
 * species (unless IONTRAP_ALLOW_UNSTABLE).  Synchronous: waits for the handle's queued
 * work first.  Handles advanced by iontrap_step_many use the new forces as well. */
int iontrap_set_params(iontrap_t *h, const iontrap_params *p, const iontrap_cooling *cooling);

/* Pseudopotential trap given by its secular frequencies, one set per species
 * (linearPseudoPT, Sec. 3 "Forces and fields": the pseudopotential frequencies depend on
 * Q/M, so each species gets its own).  omega[3 n_species] = (wx, wy, wz) of each species,
 * rad/s: the trap acceleration of an ion of species s is (-wx^2 x, -wy^2 y, -wz^2 z).  NULL
 * returns to the Eq. 2 pseudopotential of the handle's Mathieu parameters.  The handle must
 * carry IONTRAP_PSEUDO (EINVAL otherwise); a_n is evaluated again as by
 * iontrap_set_params.  EINVAL for non-finite or non-positive frequencies, EUNSTABLE when
 * w dt >= 2 on some axis (unless IONTRAP_ALLOW_UNSTABLE).  Synchronous. */
int iontrap_set_pseudo_frequencies(iontrap_t *h, const double *omega);

/* Minimisation (Sec. 3 "Minimisation"): damped dynamics that drives the ions to a minimum
 * of the static potential -- the trap (IONTRAP_PSEUDO, or a static trap: IONTRAP_RF_OFF;
 * EINVAL with the RF field on, whose minimum under damping is not the crystal's, as Sec. 3
 * explains) plus the Coulomb pair energy -- with no bath and no laser.  Starting at rest,
 * each iteration:
 *   1. a = Coulomb (the handle's pair kernel, in its precision form) + trap, F_i = M_i a_i;
 *      stop when |F| = sqrt(sum_i |F_i|^2) < ftol (newtons)
 *   2. v = (v.F / F.F) F when v.F > 0 (sums over all ions), else v = 0
 *   3. v += dt a; d = dt v; d and v are scaled by min(1, dmax / max_i |d_i|), so no ion
 *      moves more than dmax (m) in one iteration; x += d
 *   max_iters  iterations at most (>= 0)
 *   dt         iteration time step, s (0 = the handle's dt); keep omega dt well below 1
 *              for the stiffest trap axis
 * On return x_n is the last position, v_n = 0, a_n is evaluated again under the handle's
 * forces, and the step index is unchanged (minimisation is not time evolution).
 * *iters (may be NULL) receives the iterations that moved the ions and *fnorm (may be
 * NULL) |F| at the final positions.  Synchronous. */
int iontrap_minimize(iontrap_t *h, int64_t max_iters, double dt, double dmax, double ftol, int64_t *iters,
                     double *fnorm);

/* Mass-weighted Hessian of the static potential at the current positions (Sec. 5
 * "Normal modes of motion": the normal-mode frequencies are the square roots of its
 * eigenvalues), FP64, computed on the device:
 *   H[(3i+a) 3n + 3j+b] = d^2 V / dx_ia dx_jb / sqrt(M_i M_j),
 *   V = sum_i M_i (kx x_i^2 + ky y_i^2 + kz z_i^2)/2 + sum_{i<j} k_e Q_i Q_j / |x_i - x_j|
 * with k the trap springs of i's species (the pseudopotential, or the static RF-off trap).
 * H[9 n^2] is a host array, row-major, symmetric.  EINVAL with the RF field on,
 * IONTRAP_ETOOLARGE for n > 8192, ENOMEM if the 9 n^2 doubles cannot be allocated on the
 * device.  Synchronous. */
int iontrap_hessian(iontrap_t *h, double *H);

/* iontrap_step_record fields */
#define IONTRAP_REC_X 1u     /* positions x_s */
#define IONTRAP_REC_V 2u     /* velocities v_s */
#define IONTRAP_REC_VAVG 4u  /* velocities averaged over the last avg_steps steps */

/* evolve(N) with dump and timeAvg (Sec. 3 "Writing/reading data"): enqueue n_steps steps
 * and, after every `every` steps (the dump interval), write a record of the state s
 * reached to d_out.  A record holds, in this order, the fields requested:
 *   IONTRAP_REC_X     x_s [3n]
 *   IONTRAP_REC_V     v_s [3n]
 *   IONTRAP_REC_VAVG  (1/W) sum_{m=s-W+1..s} v_m [3n], W = avg_steps, the time average of
 *                     the velocity over the W steps ending at s (timeAvg; W = 20 steps is
 *                     one RF period at dt = T_RF/20: the secular velocity)
 * each [3][n] SoA in id order, so record k (0-based, state step0 + (k+1) every) starts at
 * d_out + k F 3n with F the number of fields.  d_out is a DEVICE array of
 * (n_steps / every) F 3n doubles owned by the caller; it must stay valid until the
 * stream reaches the last record (iontrap_sync).  The average uses
 * sum v_m = [(x_s - x_{s-W}) + (x_{s+1} - x_{s-W+1})] / (2 dt), exact for kick-drift-kick
 * Verlet (v_m is the mean of its two half-step velocities), so the step kernels do no
 * extra work; a snapshot of x_{s-W} is taken W steps before each record (the handle
 * holds 6n doubles for it).  EINVAL when every < 1, n_steps is not a multiple of every,
 * fields is empty or unknown, or avg_steps is not in [1, every] with IONTRAP_REC_VAVG.
 * Asynchronous like iontrap_step; forms and results are those of iontrap_step (the
 * steps are enqueued in chunks between records). */
int iontrap_step_record(iontrap_t *h, int64_t n_steps, int64_t every, uint32_t fields, int64_t avg_steps,
                        double *d_out);

/* Wait for the handle's stream and report device-side failures (ENONFINITE,
 * ETIMEOUT, ECUDA). */
int iontrap_sync(iontrap_t *h);

/* Synchronise, then copy out the state: x[3n], v[3n] (either may be NULL), the step
 * index *step and time *t = step dt (either may be NULL).  After a device-side failure
 * (IONTRAP_ENONFINITE, IONTRAP_ETIMEOUT) the state is still copied out -- for a timeout in
 * the row-persistent form it is the state the failed launch started from -- and the
 * sticky status is returned. */
int iontrap_state(iontrap_t *h, double *x, double *v, int64_t *step, double *t);

/* Synchronise, then write the Coulomb acceleration k_e e^2 z_i/M_i sum_j z_j d_ij/r_ij^3
 * at the current positions x_n into acc[3n] (SoA), computed by the handle's force
 * kernel in its precision form.  Zeros when IONTRAP_COULOMB_OFF is set. */
int iontrap_forces(iontrap_t *h, double *acc);

/* Checkpoint: synchronise, then copy out the full state x_n[3n], v_n[3n], a_n[3n]
 * (any may be NULL) and the step index.  Together with iontrap_restore it resumes a run
 * bit for bit (the paper only dumps x and v, Sec. 3 "Writing/reading data"; a_n is
 * needed too because the Langevin drag of a_n used v_{n-1/2}, not v_n). */
int iontrap_checkpoint(iontrap_t *h, double *x, double *v, double *a, int64_t *step);

/* Restore: overwrite the state of a handle with a checkpoint (x, v, a: 3n each, all
 * required; step >= 0) taken from a simulation with the same ions and parameters.
 * Synchronous.  EINVAL on NULL or non-finite input; the handle's sticky status
 * otherwise. */
int iontrap_restore(iontrap_t *h, const double *x, const double *v, const double *a, int64_t step);

/* Enqueue n_steps[k] steps on each of count handles (the batched form of evolve(N)).
 * FP32-form handles with n <= 2048 on the device of the first such handle are advanced
 * together, up to 1000 steps per launch, with every ensemble resident in shared memory
 * (positions) and registers (FP64 state): ensembles above 256 ions by groups of 2, 4 or
 * 8 CTAs of a cluster (part-major, positions exchanged through distributed shared
 * memory), smaller ones by a CTA or a warp each, the two grids side by side; the others
 * are stepped one by one as by iontrap_step.  Work is ordered after what is already queued
 * on each handle's stream, and each handle's later work waits for the batch.  A
 * batched ensemble's result depends only on its own inputs: it is bitwise the same
 * alone or in any mix (its summation order differs from iontrap_step's, so the two
 * agree to the FP32 force tolerance, not bit for bit).  Returns the first failing
 * handle's status.  The launch runs on the stream of the first batched handle; the
 * library keeps a set of launch tables for each of the last 16 streams used, so calls on
 * different streams run side by side (a 17th stream waits for the least recently used
 * set's launches), and calls on one stream are ordered. */
int iontrap_step_many(iontrap_t *const *hs, const int64_t *n_steps, int count);

/* Free the handle's device memory, graph and owned stream.  NULL is a no-op. */
void iontrap_destroy(iontrap_t *h);

/* The linear Paul trap given by its voltages and geometry, linearPT(V0, U0, R0, Z0,
 * kappa, Omega) of Sec. 3 "Forces and fields": the field of Eq. 1 expressed through the
 * Mathieu parameters of Eq. 3 for species0 (charge Q, mass M):
 *   q = 2 Q V0 / (M R0^2 Omega^2),   omega_z^2 = 2 Q kappa U0 / (M Z0^2),   a = 0.
 * Eq. 3's a_x = -4 Q kappa U0 / (M Z0^2 Omega^2) is the radial defocusing of the axial dc
 * field, which this library's trap already applies as +omega_z^2/2 (iontrap_params.a is an
 * extra dc term on top of it), so a is set to 0.  The dc field is taken as confining along
 * z: Eq. 1 prints kappa U0/Z0^2 (2z, -x, -y), which pushes a positive ion away from the
 * centre along z, while Eq. 3 gives a_z > 0 (confinement) for Q kappa U0 > 0.
 *   V0, U0    ac amplitude and dc (endcap) voltage, V
 *   R0, Z0    radial and axial characteristic lengths, m (> 0)
 *   kappa     geometric factor of the dc field
 *   Omega     RF angular frequency, rad/s (> 0)
 * Writes p->Omega, p->a, p->q and p->omega_z and leaves the other fields as they are.
 * EINVAL on non-finite or non-positive lengths / Omega / mass, or Q kappa U0 < 0 (the dc
 * field would not confine along z).  Host only. */
int iontrap_linear_pt(double V0, double U0, double R0, double Z0, double kappa, double Omega,
                      const iontrap_species *species0, iontrap_params *p);

/* Static description of a status code. */
const char *iontrap_strerror(int status);

/* Host-only check used by iontrap_create: *is_stable = 1 when every species' single-ion
 * motion is bounded under the discrete kick-drift-kick map (one-RF-period monodromy
 * |trace| < 2 along x and y; |2 - dt^2 omega_z^2| < 2 along z).  EINVAL on bad
 * arguments.  No device work. */
int iontrap_stable(const iontrap_species *species, int n_species, const iontrap_params *p,
                   int *is_stable);

/* Test hook: the device noise generator.  For each ids[k] writes the three normals of
 * (seed, counter, ids[k]) to z[3m] (SoA) as the given precision form computes them
 * (FP32 Box-Muller for IONTRAP_PREC_FP32, FP64 for IONTRAP_PREC_FP64).  Host arrays;
 * synchronous. */
int iontrap_normals(uint64_t seed, int64_t counter, const int64_t *ids, int64_t m,
                    int precision, double *z);

/* Launch configuration of a handle's step kernels. */
typedef struct {
    int32_t threads;          /* CTA size of the force kernel (64, 128, 256) */
    int32_t ions_per_thread;  /* ions held in registers per thread (1, 2, 4) */
    int32_t packed;           /* 1: the FP32 pair arithmetic runs on packed FP32x2 instructions,
                                 two ions per instruction; bitwise identical to 0 */
    int32_t jsplit;           /* j-range per CTA: grid.y = ceil(n / jsplit) */
    int32_t fused;            /* how the split partials are merged and integrated:
                                 1: by the last CTA of each i-block (arrival counter);
                                 0: by a separate epilogue kernel over all SMs;
                                 2: the splits of an i-block form a thread-block cluster
                                    (at most 8 splits; 16 in form 3) and merge through distributed shared
                                    memory, each CTA integrating a slice of the i-block;
                                 3: as 2, with an i-block of 32*ions_per_thread ions held by
                                    every warp of the CTA (threads = 32 W) and the W warps
                                    splitting the CTA's j-range into interleaved chunks;
                                 4: grid-persistent: one cooperative launch runs up to 1000
                                    steps with every CTA resident (threads = 256 or 512,
                                    ions_per_thread = 2, packed = 1; S = ceil(n / jsplit) >= 7
                                    j-segments; the (ceil(n / (2 threads)) groups x S) CTAs
                                    must fit on the GPU at once, segments at most 4096 ions);
                                    each CTA sums a group of 2*threads ions against one
                                    segment and integrates an equal share of its group; no
                                    CUDA graph, pdl ignored; not with IONTRAP_COULOMB_OFF.
                                 5: row-persistent: one cooperative launch runs up to 1000
                                    steps (threads = 256 or 512, ions_per_thread = 1 or 2,
                                    packed = 1, jsplit = R ions per CTA with 3 R <= threads,
                                    ceil(n / R) CTAs resident at once, all n positions staged
                                    in shared memory: n up to about 7000); each CTA sums its R
                                    ions over every j, thread t taking ion t % R against j-part
                                    t / R (with two ions per thread the ions s and s + RT,
                                    RT = ceil(R/2), s = t % RT, against part t / RT: every j
                                    read from shared memory serves two pairs), merges the
                                    part partials in shared memory and
                                    integrates; one grid-wide counter per step; after a
                                    launch's first step the positions arrive by bulk TMA
                                    copies of a part-major global copy that the owners
                                    write (kept in the handle's partial-sum scratch); the evaluation
                                    at creation uses form 1 over 512-ion j-ranges; not with
                                    IONTRAP_COULOMB_OFF.
                                 Form 5 gives results within the FP32 tolerances of the other
                                 forms, bitwise reproducible for a given shape.
                                 The FP64 form supports 1 only. */
    int32_t pdl;              /* 1: consecutive step kernels use programmatic dependent launch
                                 (default 0: measured slower on GB300 for these grids) */
    int32_t graph;            /* 1: iontrap_step enqueues CUDA graphs of 100 steps; 0: single launches */
} iontrap_config;

/* iontrap_get_config reads a handle's configuration; iontrap_set_config changes it (the
 * autotuner's knob).  EINVAL for a combination without a compiled kernel, jsplit < 1 or
 * > n, jsplit > 2048 in the FP64 form, more than 64 splits when not fused, or more than
 * 8 (form 2) or 16 (form 3, a non-portable cluster size) splits in the cluster forms.  Results depend only on n, the i-block (threads *
 * ions_per_thread; 32 * ions_per_thread and the warp count in form 3), jsplit and the
 * parameters: forms 0, 1 and 2 with equal values give bitwise equal trajectories. */
int iontrap_get_config(const iontrap_t *h, iontrap_config *cfg);
int iontrap_set_config(iontrap_t *h, const iontrap_config *cfg);

/* The configuration a handle of n ions in the given precision form, with the given
 * IONTRAP_* flags, starts with on the current device when no autotuned entry applies.
 * allow_persistent = 0 excludes the persistent forms (fused = 4 and 5): the serving loop
 * gives that configuration to the requests the batched kernel does not take, which it
 * steps on shared streams beside the batches, since a cooperative grid holding every SM
 * would serialise against them.  EINVAL for
 * n < 1 or an unknown precision; ECUDA without a device. */
int iontrap_default_config(int64_t n, int precision, uint32_t flags, int allow_persistent, iontrap_config *cfg);

/* Device memory held by a handle, in bytes (state, pair streams, partials, counters),
 * and the bytes a handle of n ions in the given precision form would hold when created
 * now on the current device (its default configuration, Coulomb term on); the latter does
 * no device work. */
int iontrap_device_bytes(const iontrap_t *h, int64_t *bytes);
int iontrap_estimate_bytes(int64_t n, int precision, int64_t *bytes);

/* ---------------------------------------------------------------- serving loop
 * Continuous batching of many trap simulations of different sizes and step budgets on
 * one device.  Requests wait in arrival order until a slot and enough of the device
 * memory budget are free, then stay resident until their last step.  Each
 * iontrap_server_poll is one scheduling round: retire requests whose last chunk
 * finished (final state copied to the host, memory returned), admit waiting requests
 * that fit (each created on the server's own stream, so admission does not wait for
 * chunks in flight), and enqueue the next chunks -- FP32-form requests with n <= 2048
 * through the batched kernel, chunk_steps steps of every idle one, one launch per size
 * class (up to 64, 256, 512, 1024, 2048 ions) on a stream of its own, smaller classes at
 * higher stream priority, so that a small request's chunk does not wait for a large
 * one's; the others on max_parallel shared streams, each idle stream taking the request
 * with the least remaining pair work (n^2 x steps left), in chunks of at most
 * chunk_steps x (4096 / n)^2 steps (at least one).  Handle memory comes from the
 * library's stream-ordered pool, so admission and retirement do not synchronise the
 * device.  A request's result does not depend on what else is resident (batched ones are
 * bitwise independent of the mix, the others are stepped one chunk at a time).  Poll is
 * non-blocking except for the host copies of admission and retirement.  A server and its
 * requests are used from one host thread. */
typedef struct iontrap_server iontrap_server_t;
typedef struct {
    int64_t mem_budget_bytes; /* device bytes resident requests may hold; 0 = 2 GiB */
    int32_t max_resident;     /* resident request limit; 0 = 4096 */
    int32_t chunk_steps;      /* steps per request per scheduling round; 0 = 100 */
    int32_t max_parallel;     /* shared streams of the requests the batched kernel does not
                                 take (each steps one request at a time); 0 = 3 */
} iontrap_server_config;
typedef struct {
    int64_t waiting, resident, completed, device_bytes;
} iontrap_server_counters;

int iontrap_server_create(const iontrap_server_config *cfg, iontrap_server_t **out);
/* Queue a request (arguments as for iontrap_create with step0 = 0, plus its step
 * budget); the inputs are copied.  *id identifies it in poll and result. */
int iontrap_server_submit(iontrap_server_t *s, const iontrap_species *species, int n_species,
                          const uint8_t *species_of_ion, const double *x0, const double *v0, int64_t n,
                          const iontrap_params *p, int64_t n_steps, int64_t *id);
/* One scheduling round; writes the ids completed in this round (up to cap) and their
 * count.  A request that cannot be created (e.g. IONTRAP_EUNSTABLE) completes at once
 * with that status. */
int iontrap_server_poll(iontrap_server_t *s, int64_t *completed_ids, int64_t cap, int64_t *n_completed);
/* Copy a completed request's final x[3n], v[3n] (either may be NULL), step index and
 * status, and release it.  EINVAL if the id is not completed (or already released). */
int iontrap_server_result(iontrap_server_t *s, int64_t id, double *x, double *v, int64_t *step, int *status);
int iontrap_server_stats(const iontrap_server_t *s, iontrap_server_counters *out);
/* Waits for in-flight work, frees every resident request and the server. */
void iontrap_server_destroy(iontrap_server_t *s);

/* Allocation-free Coulomb accelerations, for callers that cannot call cudaMalloc (a
 * process whose memory pool owns all device memory, a host that loads this library as a
 * plugin and owns every buffer, a loop that cannot afford cudaMalloc's implicit
 * synchronisation).  The paper has no counterpart: it is a deployment variant of the
 * force evaluation that iontrap_forces performs on a handle.
 *   species[n_species]    host species table, as for iontrap_create
 *   d_species_of_ion[n]   DEVICE array of species indices
 *   d_x[3n]               DEVICE positions, SoA, metres
 *   d_acc[3n]             DEVICE output: k_e e^2 z_i/M_i sum_j z_j (x_i - x_j)/r_ij^3
 *   cuda_stream           stream to enqueue on (NULL: legacy default stream)
 * Asynchronous: the result is ready when the stream reaches it.  Allocates nothing: the
 * pair stream, split partials and counters live in one fixed device array that is part
 * of the library image (2.25 MiB on every GPU that loads the library, held until the
 * process exits).  n > 8192 returns IONTRAP_ETOOLARGE and launches nothing.  The array's
 * device address is looked up (cudaGetSymbolAddress, with the device current) on every
 * call made outside stream capture, so calls after a cudaDeviceReset find the array
 * where the new context put it; a call made while its stream is being captured reuses
 * the address of the last uncaptured call on that device, so make one call before any
 * capture (and again after a reset).  All calls on a device share the array and each
 * clears its counters before launching: calls whose work overlaps on the GPU race and
 * must be serialised by the caller.  d_acc is set to NaN before the kernels run; an ion
 * whose sum did not complete (a bounded device wait expired) is left NaN, which is how
 * this call reports a device-side failure.  EINVAL on bad arguments, ECUDA when a launch
 * fails. */
int iontrap_forces_noalloc(const iontrap_species *species, int n_species, const uint8_t *d_species_of_ion,
                           const double *d_x, int64_t n, double *d_acc, void *cuda_stream);

/* Test hook of the failure detection (no counterpart in the paper).  Every wait of the persistent forms 4 and 5
 * -- a CTA's poller waiting for the other CTAs' arrivals on a step or group counter, a
 * CTA waiting for its bulk copies -- gives up after a time limit, sets the handle's
 * timeout flag and ends the launch, which the host reads as IONTRAP_ETIMEOUT.  This hook
 * makes that happen on purpose, with no fault and no unbounded wait: the persistent
 * launches of the handle that follow use a limit of wait_limit_ns (0 restores the default,
 * 2 s), and when cta >= 0, CTA number cta withholds its arrival on the grid-wide step
 * counter at step `step` (counted from 0 within each launch) -- a counter value nothing
 * will reach -- so that every other CTA's wait for the next step expires after the
 * limit.  The launch then stops, the handle's status becomes IONTRAP_ETIMEOUT (sticky)
 * and its step index is not advanced; in form 5 the FP64 state is the one the launch
 * started from, in form 4 it may hold some of the launch's steps.  cta < 0 turns the stall
 * off.  Synchronous (waits for queued work).  EINVAL when the handle is not in form 4 or
 * 5, when its launch has a single CTA (form 5 up to 170 ions: no cross-CTA wait), or when
 * cta is not below the launch's CTA count. */
int iontrap_test_stall(iontrap_t *h, int64_t wait_limit_ns, int32_t cta, int64_t step);

/* Profiling hook: run ONE step with per-CTA phase timestamps (%globaltimer, ns) and copy
 * them to marks[cap] (EINVAL in the grid-persistent form 4; in the row-persistent form 5
 * one launch of 8 steps, 4 marks per CTA and step at mark (CTA 8 + step) 4 + m: grid
 * barrier passed, thread 0's j-part in shared memory (its copy run landed; in the
 * launch's first step, every part staged), every pair loop done, integration done;
 * *n_force = 32 x CTAs, *n_epi = 0).  Layout: 4 marks per force-kernel CTA, CTA id = y*grid.x + x
 * (start after the grid dependency wait, end of the pair loop, start of the fused
 * epilogue or 0, end of the fused epilogue or 0), then 2 per epilogue-kernel CTA (start,
 * end) when the configuration is not fused.  *n_force and *n_epi receive the counts.
 * Synchronous; EINVAL if cap is too small. */
int iontrap_trace_step(iontrap_t *h, unsigned long long *marks, int64_t cap, int64_t *n_force, int64_t *n_epi);

/* Autotuner.  Times candidate launch configurations (threads x ions per thread x packed,
 * a ladder of split counts, the merge forms 0-3 and shapes of the persistent forms 4 and
 * 5; see iontrap_config) on this handle's own workload,
 * each for about trial_us of steps in each of two passes (a candidate's faster time
 * counts), installs the fastest and records it in the
 * process-wide tuning table under (precision, floor(log2 n)) for the current device;
 * handles created later with n in that bucket start from it.  The handle's state is
 * checkpointed before and restored after, so tuning does not advance the simulation.
 * *best and *best_us_per_step (either may be NULL) receive the winner.  Synchronous. */
typedef struct {
    int32_t precision;        /* IONTRAP_PREC_* */
    int32_t log2n;            /* bucket: floor(log2 n) */
    int32_t threads, ions_per_thread, packed, splits, fused, pdl, graph;
    float us_per_step;        /* measured time of the winner */
} iontrap_tuning_entry;
int iontrap_autotune(iontrap_t *h, double trial_us, iontrap_config *best, double *best_us_per_step);

/* iontrap_tuning_entry.precision of the batched launch's entries: the part-major groups
 * (256 < n <= 2048) of ensembles in bucket log2n use splits CTAs per group (2, 4 or 8, with
 * at most 256 ions per CTA) and ions_per_thread j-parts per CTA (0: the launcher's cost
 * model); threads = 256, fused = 6. */
#define IONTRAP_TUNE_BATCHED 2

/* Autotuner of the batched launch (iontrap_step_many, the batched form of evolve(N) of
 * Sec. 3 "Time evolution").  For every N bucket floor(log2 n) of the part-major groups among
 * the given handles (FP32 form, 256 < n <= 2048), largest bucket first, times one batched
 * launch of all count handles under each candidate shape of that bucket -- CTAs per group
 * C in {2, 4, 8} and j-parts NP in {cost model, 2, 4, 6, 8, 12}, as far as they fit -- with
 * the buckets already tuned at their winners and the others at the launcher's defaults,
 * each candidate for about trial_us of steps in each of two passes (its faster time
 * counts), and records the winner in the tuning table under (IONTRAP_TUNE_BATCHED, bucket)
 * for the current device; later batched launches of ensembles in that bucket use it.  The
 * group shape is a function of the bucket alone, so an ensemble's result stays the same
 * alone or in any mix.  Every handle's state is checkpointed before and restored after
 * (tuning does not advance the simulations).  Synchronous. */
int iontrap_autotune_many(iontrap_t *const *hs, int count, double trial_us);
/* Read the tuning table of the current device (up to cap entries; *count = entries). */
int iontrap_tuning_get(iontrap_tuning_entry *out, int cap, int *count);
/* Add or replace entries of the current device's tuning table (e.g. saved from an
 * earlier autotuning run on the same kind of GPU); an entry with splits = 0 removes the
 * table's entry of its (precision, log2n) instead. */
int iontrap_tuning_put(const iontrap_tuning_entry *in, int count);

/* Microbenchmark of the pipes the step kernels use (not part of the method): runs
 * independent dependency chains of one instruction kind on every SM of the current
 * device and reports lane operations per SM clock and the SM clock seen.
 * kind: 0 FFMA, 1 packed FFMA2 (2 lanes each), 2 MUFU rsqrt, 3 DFMA, 4 packed FADD2,
 * 5 FP32 <-> FP64 conversions (lane operations = conversions). */
int iontrap_alu_probe(int kind, long long iters, double *lane_ops_per_clk_per_sm, double *sm_mhz);

#ifdef __cplusplus
}
#endif

#endif /* IONTRAP_H */
