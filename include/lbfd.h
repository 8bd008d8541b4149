/*
 * lbfd.h -- C ABI of the GB300 fluctuating lattice-Boltzmann diffusion library.
 *
 * The method is the fluctuating lattice-Boltzmann scheme for the diffusion
 * equation of Wagner & Strand (arXiv:1606.07801):
 *   f_i(x + v_i, t + 1) = f_i(x, t) + Omega_i                       (eq. LB)
 *   Omega_i = sum_j Lambda_ij (f^0_j - f_j) + xi_i           (eq. collision)
 * with f^0_i = rho w_i (eq. f0def), single relaxation time Lambda = 1/tau
 * (eq. coll), and noise xi^a in the non-conserved moments of a weighted
 * orthonormal basis with variance rho (2 tau - 1)/tau^2 (eq. xiglobal with
 * the global density rho^eq, eq. xilocal with the local density, which is
 * clamped at zero as in Sec. IV).  Streaming is periodic.
 *
 * State convention.  The populations a caller sees (lbfd_get_f, lbfd_set_f,
 * lbfd_moments, lbfd_observables) are the paper's f_i(x, t): the values
 * that enter the collision at step t.  Internally the library keeps the
 * post-collision values of the previous step, g_i(x) = f_i(x + v_i, t)
 * (the pull scheme's natural state); the entry points above convert with an
 * exact streaming shift through the spare buffer.
 *
 * Every entry point returns LBFD_OK (0) or a negative status; none aborts the
 * process.  lbfd_last_error() returns a message for the calling thread's
 * last failure.  A handle may be used by one host thread at a time.
 * Pointers named *_host are host memory (pageable or pinned); pointers named
 * *_dev are device memory of the handle's device.  The library never frees
 * memory it did not allocate.
 */
#ifndef LBFD_H
#define LBFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBFD_ABI_VERSION 1

/* ---- status codes ---------------------------------------------------- */
#define LBFD_OK 0
#define LBFD_EINVAL (-1)   /* bad argument (unknown lattice, dim < 1, tau <= 1/2, rho_mean < 0, n < 0, ...) */
#define LBFD_ENOMEM (-2)   /* a device or host allocation failed */
#define LBFD_ECUDA (-3)    /* a CUDA call failed; lbfd_last_error() names it */
#define LBFD_ETIMEOUT (-4) /* a bounded device wait gave up */
#define LBFD_EBUSY (-5)    /* the resource is in use */
#define LBFD_ENOTSUP (-6)  /* valid but not supported by this build */

/* ---- lattices (velocity order is part of the ABI: f is stored [i][site]) -- */
#define LBFD_D1Q3 0  /* v = 0, +1, -1;  w = 2/3, 1/6, 1/6 */
#define LBFD_D2Q9 1  /* v = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9 x4, 1/36 x4 */
#define LBFD_D3Q19 2 /* v = 0; (+-1,0,0),(0,+-1,0),(0,0,+-1) as +x,-x,+y,-y,+z,-z;
                        (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0); (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1);
                        (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1);  w = 1/3, 1/18 x6, 1/36 x12 */
#define LBFD_D2Q5 3  /* the paper's lattice (Sec. II): v = (0,0),(1,0),(-1,0),(0,1),(0,-1);
                        w = 1 - 2 theta, theta/2 x4 with free theta in (0, 1/2); basis by
                        Gram-Schmidt of 1, v_x, v_y, v_x^2 - v_y^2, v_x^2 + v_y^2.  FP32/FP64 only;
                        not in ensembles or the server */

/* ---- arithmetic and storage ------------------------------------------ */
#define LBFD_F32 0      /* FP32 arithmetic and storage (default) */
#define LBFD_F64 1      /* FP64 arithmetic and storage */
#define LBFD_F32_F16 2  /* FP32 arithmetic; f_i - w_i rho_mean stored as IEEE binary16 (round to nearest even) */
#define LBFD_F32_BF16 3 /* FP32 arithmetic; f_i - w_i rho_mean stored as bfloat16 (round to nearest even) */

/* ---- noise ------------------------------------------------------------- */
#define LBFD_NOISE_LOCAL 0  /* variance from the local density, clamped at 0 (eq. xilocal) */
#define LBFD_NOISE_GLOBAL 1 /* variance from rho^eq = rho_mean, the conserved mass per site (eq. xiglobal) */
#define LBFD_NOISE_OFF 2    /* deterministic lattice-Boltzmann diffusion */
#define LBFD_GAUSSIAN 0     /* unit normals (Box-Muller on Philox4x32-10 words) */
#define LBFD_UNIFORM 1      /* unit-variance flat variates on (-sqrt3, sqrt3) (Sec. IV) */

/* ---- initial state ------------------------------------------------------ */
#define LBFD_INIT_UNIFORM 0 /* f_i = w_i rho_mean */
#define LBFD_INIT_SINE 1    /* f_i = w_i (rho_mean + sine_amp sin(2 pi (kx x/Lx + ky y/Ly + kz z/Lz))) */
#define LBFD_INIT_NONE 2    /* contents undefined until lbfd_set_f */

#define LBFD_MAX_Q 19
#define LBFD_MAX_MODES 16

/* ---- step kernels (lbfd_options.step_kernel, lbfd_step_kernel) ---------------
 * Every kernel computes the same site update with the same arithmetic, so the
 * choice changes speed only, never a result bit. */
#define LBFD_KERNEL_AUTO 0    /* the library's choice (option value only) */
#define LBFD_KERNEL_VEC 1     /* k_step_vec: two or four sites of a row per thread, pulled straight from
                                 global memory (Lx even); FP32-arithmetic formats collide two sites at a time
                                 on the packed FP32 instructions where that is faster, with the same result */
#define LBFD_KERNEL_SCALAR 2  /* k_step: one site per thread (any Lx) */
#define LBFD_KERNEL_SMALL 3   /* k_step_small: many steps per launch in one block's shared memory (small
                                 lattices, n >= 2; chosen automatically) */
#define LBFD_KERNEL_CLUSTER 4 /* k_step_cluster: the same over a thread-block cluster (chosen automatically) */
#define LBFD_KERNEL_MRT 5     /* k_step_mrt: moment-space collision (D2Q5, multiple relaxation times) */
#define LBFD_KERNEL_STAGED 6  /* k_step_staged: persistent; each tile's source rows are copied into shared
                                 memory by the TMA unit (bulk asynchronous copies on an mbarrier), the sites
                                 pull from there, and the results go back by bulk stores.  Needs
                                 Lx * (bytes per stored value) to be a multiple of 16 and 16-byte aligned
                                 buffers; D1Q3, D2Q9, D3Q19 */

/* Options of lbfd_create_ex.  Fill with lbfd_options_init, then override. */
typedef struct lbfd_options {
    int32_t lattice;    /* LBFD_D1Q3 / LBFD_D2Q9 / LBFD_D3Q19 */
    int32_t precision;  /* LBFD_F32 / LBFD_F64 / LBFD_F32_F16 / LBFD_F32_BF16 */
    int32_t noise_mode; /* LBFD_NOISE_* */
    int32_t noise_dist; /* LBFD_GAUSSIAN / LBFD_UNIFORM */
    int32_t init;       /* LBFD_INIT_* */
    int32_t device;     /* CUDA device ordinal; -1 = the calling thread's current device */
    int64_t dims[3];    /* Lx, Ly, Lz (x fastest); trailing dims of lower-D lattices must be 1 */
    double tau;         /* relaxation time, > 1/2 */
    double rho_mean;    /* mean density per site, >= 0 */
    double sine_amp;    /* amplitude for LBFD_INIT_SINE */
    int32_t sine_k[3];  /* integer wave vector for LBFD_INIT_SINE */
    uint32_t lattice_id; /* Philox counter word 1: distinguishes lattices sharing a seed */
    uint64_t seed;      /* Philox key */
    void *stream;       /* cudaStream_t the handle works on; NULL = legacy default stream */
    void *f_dev[2];     /* optional caller-owned device buffers, each Q*N values of the
                           storage format; both or neither.  Never freed by the library. */
    int32_t n_modes;    /* structure-factor wave vectors sampled by lbfd_sample */
    int32_t modes[LBFD_MAX_MODES][3];
    int32_t step_kernel; /* LBFD_KERNEL_AUTO, or LBFD_KERNEL_VEC / LBFD_KERNEL_SCALAR /
                            LBFD_KERNEL_STAGED to ask for that kernel for the one-launch-per-step path
                            (LBFD_EINVAL where the lattice does not meet its requirements).  Small
                            lattices still take the many-steps-per-launch path. */
    int32_t wait_test_bytes; /* tests of the staged kernel's bounded waits only (0 in normal use): every
                            CTA's first tile waits for this many bytes more than its copies deliver, so
                            the wait runs out after about a second, the kernel stops, and the next
                            synchronous call reports LBFD_ETIMEOUT.  Needs the staged kernel; < 2^20 */
    int32_t slab_global; /* slab decomposition of one lattice over several processes (see
                            lbfd_slab_bounds); 0 = the handle holds the whole lattice.  > 0: the lattice
                            has slab_global planes along its slowest axis (y for D2Q9, z for D3Q19) and
                            this handle owns planes slab_first .. slab_first + n - 1, n = that axis'
                            entry of dims (the other dims are the whole lattice's).  The handle stores
                            n + 2 planes, a halo plane on each side, and keys the noise of a site by its
                            global index.  Between steps the caller fills the halo planes of the current
                            state (lbfd_state_device) with its neighbours' crossing populations
                            (lbfd_slab_halo).  Slab handles take one step per lbfd_step call, run the
                            staged kernel (LBFD_ENOTSUP where it cannot run), and offer no mass or
                            sampling; lbfd_set_f(_raw) take the owned planes plus both halo planes
                            (n + 2 planes), the other readers return the owned planes. */
    int32_t slab_first;
    int32_t sample_every; /* s > 0: lbfd_step also adds the observables of f(x, t) to the accumulators
                            (as lbfd_sample would) at every step t with t mod s == 0, before that
                            step's collision.  For the FP32-arithmetic formats with at most 4
                            modes this runs inside the step kernel (one pass over the state);
                            otherwise lbfd_step runs the separate pass first.  0 = off */
    int32_t reserved[3];
    double theta;       /* D2Q5: sum_i w_i v_ix^2, in (0, 1/2); 0 = 1/3.  Other lattices: 0 or 1/3 */
    double tau_moments[LBFD_MAX_Q]; /* multiple relaxation times (Sec. III): tau^a of moment a of
                           the basis, a = 1..Q-1 (entry 0, the conserved density, is ignored);
                           0 = tau.  Each moment's noise variance is rho (2 tau^a - 1)/(tau^a)^2.
                           Any entry other than 0 or tau selects the moment-space kernel
                           (FP32/FP64 storage, Q * sites < 2^32). */
} lbfd_options;

/* Observables accumulated by lbfd_sample (FP64, deterministic reductions). */
typedef struct lbfd_obs {
    int64_t t;         /* steps taken since creation (or the last lbfd_set_t) */
    int64_t n_samples; /* lbfd_sample calls since creation or lbfd_reset_obs */
    int32_t Q, n_modes;
    double sum_rho;    /* sum over samples of sum_x rho(x) */
    double sum_rho2;   /* sum over samples of sum_x rho(x)^2 */
    double sum_f[LBFD_MAX_Q];              /* sum over samples of sum_x f_i(x) */
    double sum_ff[LBFD_MAX_Q * LBFD_MAX_Q]; /* sum over samples of sum_x f_i(x) f_j(x), [i*Q + j] */
    double sum_sk[LBFD_MAX_MODES];         /* sum over samples of |sum_x (rho(x) - rho_mean) e^{-2 pi i k.x/L}|^2 */
} lbfd_obs;

typedef struct lbfd_sim *lbfd_t;

/* Fills *opt with defaults: D2Q9, FP32, local Gaussian noise, uniform start,
 * dims 1, tau 1, rho_mean 1, seed 1, current device, legacy default stream. */
int lbfd_options_init(lbfd_options *opt);

/* Creates a simulation (the boundary named in the method: lattice, dims, tau,
 * rho_mean, seed) with FP32 arithmetic, local Gaussian noise and a uniform
 * start f_i = w_i rho_mean.  dims has D entries (D = 1, 2, 3 for D1Q3, D2Q9,
 * D3Q19).  Allocates two Q*N device buffers on the current device. */
int lbfd_create(lbfd_t *out, int32_t lattice, const int64_t *dims, double tau, double rho_mean,
                uint64_t seed);

/* Creates a simulation from a full option set (see lbfd_options). */
int lbfd_create_ex(lbfd_t *out, const lbfd_options *opt);

/* Frees what the handle allocated; caller-owned buffers are left alone.
 * Synchronises the handle's stream first.  NULL is accepted. */
int lbfd_destroy(lbfd_t h);

/* Advances the state by n >= 0 steps of eq. LB (collide, add noise,
 * stream).  Asynchronous on the handle's stream; t advances by n. */
int lbfd_step(lbfd_t h, int64_t n);

/* Sets lbfd_options.sample_every of a handle (0 turns the sampling in
 * lbfd_step off).  LBFD_EINVAL for a slab handle or every < 0. */
int lbfd_set_sample_every(lbfd_t h, int32_t every);

/* The kernel lbfd_step(h, n) would run for this n (one of LBFD_KERNEL_VEC ..
 * LBFD_KERNEL_MRT), into *kernel.  No device work. */
int lbfd_step_kernel(lbfd_t h, int64_t n, int32_t *kernel);

/* ---- slab decomposition (one lattice over several processes) -------------
 * The step of eq. LB reads nearest neighbours only, so a lattice cut into
 * slabs along its slowest axis evolves exactly as a whole if each slab holds,
 * before every step, one plane beyond each face with the populations that
 * cross it (3 for D2Q9, 5 for D3Q19).  The noise is keyed by the global site
 * index, so the split run is bit-identical to the unsplit one.  These calls
 * are host arithmetic only. */

/* Planes [*first, *first + *count) of global_planes for rank of nranks
 * (balanced; the first global_planes mod nranks ranks hold one more). */
int lbfd_slab_bounds(int64_t global_planes, int32_t nranks, int32_t rank, int64_t *first, int64_t *count);

/* Populations with velocity component dir (+1 or -1) along the slowest axis
 * (the ones that cross a face in that direction), in velocity order, into
 * pops (may be NULL) and their number into *n_pops.  D2Q9 and D3Q19. */
int lbfd_slab_cross(int32_t lattice, int32_t dir, int32_t *pops, int32_t *n_pops);

/* Exchange plan of one face of a slab whose dims are as in lbfd_options
 * (dims of the slowest axis = owned planes n): value offsets, within the
 * slab's state buffer (lbfd_state_device, n + 2 stored planes), of the
 * *n_pops planes of *plane_values values that this slab sends through the
 * face (send_off) and of the halo planes it receives into (recv_off), in
 * matching order.  face 0 is the low face (to and from the rank below),
 * face 1 the high face.  What one slab sends through its high face, the slab
 * above receives through its low face, in the same order.  Either offset
 * array may be NULL. */
int lbfd_slab_halo(int32_t lattice, const int64_t *dims, int32_t face, int64_t *send_off, int64_t *recv_off,
                   int32_t *n_pops, int64_t *plane_values);

/* Waits for all work queued on the handle's stream.  LBFD_ETIMEOUT if a
 * bounded device wait of a step kernel gave up since the last check (the
 * state is then not valid); lbfd_get_f, lbfd_get_f_raw, lbfd_moments,
 * lbfd_mass and lbfd_observables report it the same way. */
int lbfd_sync(lbfd_t h);

/* Step counter t; lbfd_set_t sets it (resume from a checkpoint: the noise
 * is keyed by t, so a resumed run is bit-identical to an unbroken one). */
int lbfd_get_t(lbfd_t h, int64_t *t);
int lbfd_set_t(lbfd_t h, int64_t t);

/* Copies the populations out to / in from host memory as FP64, layout
 * [i][site], site = x + Lx (y + Ly z).  Synchronous. */
int lbfd_get_f(lbfd_t h, double *f_host);
int lbfd_set_f(lbfd_t h, const double *f_host);

/* Same in the storage format (float for LBFD_F32, double for LBFD_F64, the
 * 16-bit deviation f_i - w_i rho_mean for LBFD_F32_F16 / LBFD_F32_BF16), with
 * no conversion: one cudaMemcpyAsync of Q*N values, then a stream sync.
 * Pinned host memory makes these run at full link speed. */
int lbfd_get_f_raw(lbfd_t h, void *f_host);
int lbfd_set_f_raw(lbfd_t h, const void *f_host);

/* Density rho(x) = sum_i f_i (N values) and, if j_host is not NULL, flux
 * j_a(x) = sum_i f_i v_ia (D*N values, [a][site]), FP64, to host memory.
 * Synchronous. */
int lbfd_moments(lbfd_t h, double *rho_host, double *j_host);

/* Same into caller-owned device buffers; asynchronous on the handle's stream. */
int lbfd_moments_device(lbfd_t h, double *rho_dev, double *j_dev);

/* Total mass sum_x sum_i f_i by a deterministic FP64 reduction (paper Sec.
 * IV: the mass the dynamics conserve).  For a slab handle: the FP64 sum over
 * its owned planes of the stored state, a permutation of the lattice's
 * values, so the sum of the slabs' masses over all ranks (an FP64
 * all-reduce) is the lattice's mass.  Synchronous. */
int lbfd_mass(lbfd_t h, double *mass);

/* Adds the current state's statistics to the FP64 accumulators (sums of rho,
 * rho^2, f_i, f_i f_j over sites and |rho(k)|^2 for the configured modes;
 * paper Sec. IV, eqs. rhoth, dijexp, fkfk).  Asynchronous.  Not for slab
 * handles (see lbfd_sample_totals). */
int lbfd_sample(lbfd_t h);
int lbfd_reset_obs(lbfd_t h);

/* One sample's sums over this handle's own sites, before they are combined:
 * totals[nq], nq = 2 + Q + 2 K + Q (Q + 1) / 2 (K = the handle's modes), in
 * FP64: [sum delta, sum delta^2, sum_x e_i (i < Q), (re, im) of
 * sum_x (rho - rho_mean) e^{-2 pi i k_m.x / L} (m < K), sum_x e_i e_j (i <= j,
 * row-major)], with e_i = f_i - c_i, c_i = w_i rho_mean rounded to FP32 and
 * delta = sum_i e_i.  Every entry is a sum over sites, so the totals of the
 * slabs of one lattice add up (an FP64 all-reduce over the ranks) to the
 * lattice's; the mode phases use the global site coordinates and periods.
 * For a slab handle the sites are its owned planes, whose neighbours in the
 * halo planes must be current (filled as before a step).  The state is read
 * as it stands (f(x, t)); FP32-arithmetic formats only (FP64 storage:
 * LBFD_ENOTSUP); sums in FP32 over tiles of 256 sites, FP64 beyond.
 * Synchronous; the handle's accumulators do not change. */
int lbfd_sample_totals(lbfd_t h, double *totals);

/* The accumulator entries of one sample from its (combined) totals, in the
 * layout of lbfd_obs: acc[2 + Q + Q*Q + K] = [sum rho, sum rho^2, sum f_i,
 * sum f_i f_j (Q x Q), |rho(k_m)|^2], for a lattice of n_sites sites (rho =
 * sum_i c_i + delta and f_i = c_i + e_i expanded in FP64; the squares of the
 * modes taken after the slabs are combined).  Host arithmetic only, no
 * device work. */
int lbfd_obs_restore(int32_t lattice, int32_t n_modes, double rho_mean, int64_t n_sites, const double *totals,
                     double *acc);

/* Adds one sample's accumulator entries (lbfd_obs_restore) into the handle's
 * accumulators and counts the sample: how slab handles accumulate the
 * lattice's statistics.  Synchronous. */
int lbfd_obs_add(lbfd_t h, const double *acc);

/* Reads the accumulators and the current mass.  Synchronous. */
int lbfd_observables(lbfd_t h, lbfd_obs *obs);

/* Static facts of a handle: Q, D, N (sites), bytes per stored value (8, 4 or 2). */
int lbfd_query(lbfd_t h, int32_t *Q, int32_t *D, int64_t *N, int32_t *value_bytes);

/* Device buffer holding the stored state g_i(x) = f_i(x + v_i, t) (layout
 * [i][site]; valid until the next step), and the stream the handle works on.
 * Work the handle ran on its side stream (the stage 2 of sampled steps) is
 * ordered before whatever is enqueued on that stream after this call. */
int lbfd_state_device(lbfd_t h, void **f_dev, void **stream);

/* Lattice tables the CUDA kernels use: velocities v[Q][3], weights w[Q] and
 * the moment matrix m[a][i] (Gram-Schmidt basis of Sec. II, n_i^a = m_i^a w_i).
 * Any output pointer may be NULL.  No device work. */
int lbfd_lattice_tables(int32_t lattice, int32_t *Q, int32_t *v, double *w, double *m);

/* Same for a given theta (D2Q5: weights and basis of that theta; the other
 * lattices accept only theta = 1/3 or 0). */
int lbfd_lattice_tables_ex(int32_t lattice, double theta, int32_t *Q, int32_t *v, double *w, double *m);

/* Noise variates the step kernel draws: z^1..z^nmom (unit variance) of sites
 * site0 .. site0+nsites-1 at step t, computed on the current device in the
 * given precision and returned as FP64 [site][moment] in host memory.
 * Philox4x32-10 call j has counter (site, lattice_id, t mod 2^32,
 * (t >> 32) * 8 + j) and key (seed mod 2^32, seed >> 32); moments
 * 4j+1..4j+4 take its four words.  Synchronous; allocates a temporary
 * device buffer. */
int lbfd_noise_draw(int32_t precision, int32_t dist, uint64_t seed, uint32_t lattice_id, uint64_t t,
                    int64_t site0, int64_t nsites, int32_t nmom, double *z_host);

/* Box-Muller normals the step kernel makes from given Philox words:
 * (z[2k], z[2k+1]) from (words[2k], words[2k+1]) with u = ((r >> 8) + 1/2) 2^-24,
 * z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1), computed on
 * the current device in the given precision; host arrays of 2*npairs values.
 * For checks of the edges of the uniform grid.  Synchronous; allocates
 * temporary device buffers. */
int lbfd_box_muller_probe(int32_t precision, const uint32_t *words_host, int64_t npairs, double *z_host);

/* The FP32 arithmetic of the collision on given operands, one value at a time
 * and two values per packed instruction (the step kernels collide two
 * neighbouring sites at once where that is faster, and the two forms must
 * round alike).  For k < n (n even) and the operations op = 0 add a + b,
 * 1 sub a - b, 2 mul a b, 3 fma(a, b, c), 4 (a b) + c and 5 c - (a b) (the
 * last two rounded twice), out[(2 op + form) n + k] holds the result of
 * (a[k], b[k], c[k]), form 0 computed alone and form 1 packed with value
 * k ^ 1.  Host arrays: a, b, c of n floats, out of 12 n.  Current device;
 * synchronous; allocates temporary device buffers.  LBFD_EINVAL for a null
 * array or an odd or negative n. */
int lbfd_lane_ops_probe(const float *a_host, const float *b_host, const float *c_host, int64_t n, float *out_host);

/* Total mass sum_x sum_i f_i, like lbfd_mass, for callers that cannot
 * allocate device memory: a host framework that reserved the GPU for its own
 * allocator and forbids libraries to allocate, a service under a fixed
 * device-memory budget, or a loop that cannot afford cudaMalloc/cudaFree
 * (they can synchronise the device).  The paper has no counterpart; this is
 * a library service.
 *   f_dev    device array of Q*n_sites values (float for LBFD_F32, double for
 *            LBFD_F64), layout [i][site]; any storage order of the sites works
 *            (the sum is over all of them)
 *   mass_dev caller-owned device double that receives the sum
 *   stream   cudaStream_t to launch on (NULL: legacy default stream)
 * Asynchronous; calls no cudaMalloc, cudaFree or allocating library routine.
 * Its partial sums live in a fixed 128 KiB device array that every GPU
 * loading the library holds until exit, so n_sites is limited to 16,777,216
 * (LBFD_EINVAL beyond).  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  A failed lookup is not remembered: the next call tries
 * again.  A CUDA error still pending on the calling thread from earlier work
 * is reported as LBFD_ECUDA before anything is launched (and cleared), so a
 * launch failure reported here is always this call's own.  Every call
 * overwrites the partials it reads, so no state
 * carries over, but all calls share the array: calls whose kernels overlap
 * on the GPU race and may return wrong sums; order them on one stream. */
int lbfd_mass_noalloc(int32_t lattice, int32_t precision, const void *f_dev, int64_t n_sites, double *mass_dev,
                      void *stream);

/* ---- batched ensembles ------------------------------------------------------
 * Many independent lattices of one lattice type (each with its own size,
 * tau, rho_mean, seed and Philox lattice id) advanced together: one launch
 * per time step covers every member, and chunks of steps are captured into a
 * CUDA graph and replayed.  Every member evolves exactly as the same lattice
 * would under lbfd_create_ex with the same parameters (same arithmetic,
 * same noise keys).  Members share one precision, noise mode and law, and
 * each member has Q * sites < 2^32.  Work decomposition: a work item is 1
 * or 2 sites of a row (2 only where Lx is even), a tile is `passes` x 256
 * items of one member, and the tiles go to blocks in one of the orders
 * LBFD_WALK_* (see lbfd_ensemble_tune / lbfd_ensemble_plan). */
typedef struct lbfd_member {
    int64_t dims[3];    /* Lx, Ly, Lz; trailing dims of lower-D lattices must be 1 */
    double tau;         /* > 1/2 */
    double rho_mean;    /* >= 0 */
    uint64_t seed;      /* Philox key */
    uint32_t lattice_id; /* Philox counter word 1 */
    int32_t init;       /* LBFD_INIT_UNIFORM / LBFD_INIT_SINE / LBFD_INIT_NONE */
    double sine_amp;
    int32_t sine_k[3];
    int32_t reserved;
} lbfd_member;

typedef struct lbfd_ens *lbfd_ens_t;

/* Creates an ensemble of n members on the current device (all populations in
 * two device buffers allocated here).  stream: a cudaStream_t other than the
 * legacy default stream (graphs are captured on it); NULL makes the ensemble
 * create and own a non-blocking stream.  The initial decomposition is two
 * sites per item where Lx is even, 4 passes, occupancy variant 0, one block
 * per tile (lbfd_ensemble_tune / lbfd_ensemble_plan change it). */
int lbfd_ensemble_create(lbfd_ens_t *out, int32_t lattice, int32_t precision, int32_t noise_mode, int32_t noise_dist,
                         const lbfd_member *members, int32_t n, void *stream);
int lbfd_ensemble_destroy(lbfd_ens_t e);

/* Advances every member by n steps (asynchronous).  Same step rule as
 * lbfd_step; t is shared by the members. */
int lbfd_ensemble_step(lbfd_ens_t e, int64_t n);
int lbfd_ensemble_sync(lbfd_ens_t e);

/* Times the candidate work decompositions (at most 1 or 2 sites per item,
 * times tiles of 1, 2, 4 or 8 passes, times two register/occupancy variants
 * of the kernel, times the four tile orders LBFD_WALK_*) over `steps`
 * launches each that write only the spare buffers, keeps the fastest and
 * reports it: sites per item at most, passes, resident blocks per SM (any
 * output may be NULL; lbfd_ensemble_query also gives the tile order).  The
 * state and t are unchanged.  Synchronous. */
int lbfd_ensemble_tune(lbfd_ens_t e, int32_t steps, int32_t *vx_chosen, int32_t *passes_chosen,
                       int32_t *blocks_per_sm);

/* Sets the work decomposition without timing: sites per item at most
 * (1 or 2), tile passes (1, 2, 4 or 8), register/occupancy variant (0 or 1)
 * and tile order (LBFD_WALK_*).  Every decomposition gives the same
 * results.  LBFD_EINVAL on any other value.  Synchronous. */
int lbfd_ensemble_plan(lbfd_ens_t e, int32_t vx_max, int32_t passes, int32_t occupancy, int32_t walk);

/* Members, total sites, t and the current decomposition: sites per item at
 * most, tile passes, resident blocks per SM, tile order LBFD_WALK_* (any
 * pointer may be NULL). */
int lbfd_ensemble_query(lbfd_ens_t e, int32_t *n_members, int64_t *total_sites, int64_t *t, int32_t *vx,
                        int32_t *passes, int32_t *blocks_per_sm, int32_t *walk);

/* Per-member state in FP64, layout [i][site] (as lbfd_get_f / lbfd_set_f),
 * and FP64 mass.  Synchronous. */
int lbfd_ensemble_get_f(lbfd_ens_t e, int32_t member, double *f_host);
int lbfd_ensemble_set_f(lbfd_ens_t e, int32_t member, const double *f_host);
int lbfd_ensemble_mass(lbfd_ens_t e, int32_t member, double *mass);

/* ---- serving: continuous batching of simulation requests ----------------
 * A server keeps many simulations resident on one GPU and advances them
 * together.  Requests (lattice, size, tau, rho_mean, seed, steps, initial
 * state, result kind) queue on submission.  Between time steps the server
 * admits queued requests, in arrival order with later ones allowed past an
 * earlier one that does not fit, while a slot is free and their two
 * population blocks fit in its device-memory budget (one arena allocated at
 * creation; admission and retirement allocate nothing).  Every time step
 * is one launch per lattice type covering all resident simulations of that
 * type (the batched kernel of the ensemble), plus one single-lattice launch
 * for each simulation of at least solo_sites sites, all on side streams, so
 * requests that arrive while others run join the next step and their work
 * overlaps on the device.  A
 * simulation that has taken its steps is read back on a second stream while
 * the others go on, and its memory returns to the arena once the copy is
 * done.  Each simulation keeps its own step counter t (from 0) and its own
 * Philox key and lattice id, so its result is bit-identical to the same
 * lattice run alone by lbfd_create_ex / lbfd_step / lbfd_get_f_raw or
 * lbfd_moments.  Members share one precision and noise mode and law.  A
 * server is used by one host thread at a time. */
#define LBFD_INIT_HOST 3    /* request only: f(x, 0) copied from in_host (storage format, [i][site]) */
#define LBFD_RESULT_F 0     /* result: f(x, t = steps) in the storage format, Q*N values [i][site] */
#define LBFD_RESULT_RHO 1   /* result: rho(x, t = steps) as N doubles */
#define LBFD_RESULT_NONE 2  /* no result copy; completion only */

#define LBFD_POLICY_FIFO 0      /* admit in arrival order (later requests may pass one that does not fit) */
#define LBFD_POLICY_SHORTEST 1  /* admit the request with the fewest site updates (sites x steps) first */
#define LBFD_POLICY_LONGEST 2   /* admit the request with the most site updates first: a backlog ends with
                                   fewer long simulations running alone (a shorter makespan), at the cost of
                                   the short requests' latency */
/* Tile order of the batched kernel: a persistent grid whose blocks take every
 * grid-th tile (STRIDED) or one run of consecutive tiles (CONTIGUOUS); one
 * block per tile (PER_TILE); or one block per tile with the members'
 * arguments in the kernel parameters, one launch per group of up to 112
 * members (PARAM).  Results do not depend on it. */
#define LBFD_WALK_STRIDED 0
#define LBFD_WALK_CONTIGUOUS 1
#define LBFD_WALK_PER_TILE 2
#define LBFD_WALK_PARAM 3

#define LBFD_REQ_UNKNOWN (-1)
#define LBFD_REQ_QUEUED 0
#define LBFD_REQ_RUNNING 1  /* resident, or its result is being copied */
#define LBFD_REQ_DONE 2     /* result written to the host */

typedef struct lbfd_server_options {
    int32_t precision;      /* LBFD_F32 (default) / LBFD_F64 / LBFD_F32_F16 / LBFD_F32_BF16 */
    int32_t noise_mode;     /* LBFD_NOISE_* */
    int32_t noise_dist;     /* LBFD_GAUSSIAN / LBFD_UNIFORM */
    int32_t device;         /* CUDA device ordinal; -1 = current */
    int64_t hbm_budget;     /* bytes of the device arena for resident states (allocated at creation) */
    int64_t max_active_sites; /* admit only while resident sites stay <= this (0 = no limit) */
    int32_t max_active;     /* simulations resident at once (<= 65536) */
    int32_t max_ahead;      /* time steps the host may queue ahead of the GPU (>= 1) */
    int32_t passes;         /* tile passes of the batched kernel: 1, 2, 4 or 8 */
    int32_t policy;         /* LBFD_POLICY_FIFO / LBFD_POLICY_SHORTEST / LBFD_POLICY_LONGEST */
    int32_t occupancy;      /* register/occupancy variant of the batched kernel: 0 or 1 (fewer blocks per SM) */
    int32_t walk;           /* tile order of the batched kernel: LBFD_WALK_STRIDED, _CONTIGUOUS,
                               _PER_TILE (default) or _PARAM (the members' arguments in the kernel
                               parameters, one launch per group of up to 112 residents, regrouped
                               whenever the resident set changes) */
    int32_t vx_max;         /* sites per work item of the batched kernel at most: 2 (members with even Lx
                               take two) or 1 (a kernel without the two-site path, fewer registers) */
    int32_t reserved[5];
    int64_t solo_sites;     /* simulations of at least this many sites are stepped by their own
                               single-lattice launch (parameters as kernel arguments) instead of the
                               batched launch; 0 = all batched.  Results are the same either way. */
} lbfd_server_options;

typedef struct lbfd_request {
    int32_t lattice;        /* LBFD_D1Q3 / LBFD_D2Q9 / LBFD_D3Q19 */
    int32_t init;           /* LBFD_INIT_UNIFORM / LBFD_INIT_SINE / LBFD_INIT_HOST */
    int64_t dims[3];        /* Lx, Ly, Lz; trailing dims of lower-D lattices must be 1 */
    double tau;             /* > 1/2 */
    double rho_mean;        /* >= 0 */
    uint64_t seed;          /* Philox key */
    uint32_t lattice_id;    /* Philox counter word 1 */
    int32_t result;         /* LBFD_RESULT_* */
    int64_t steps;          /* time steps to take, >= 0 */
    double sine_amp;        /* LBFD_INIT_SINE */
    int32_t sine_k[3];
    int32_t reserved;
    const void *in_host;    /* LBFD_INIT_HOST: Q*N values; read when the request is admitted */
    void *out_host;         /* result buffer (caller-owned, written asynchronously; pinned memory
                               lets the copy overlap the GPU work, pageable memory makes the
                               host wait for it); NULL in lbfd_server_run_trace = its sink */
} lbfd_request;

typedef struct lbfd_server_stats {
    int64_t submitted, queued, running, done;
    int64_t clock;             /* time steps launched so far */
    int64_t site_updates;      /* sum of sites x steps over finished requests */
    int64_t resident_bytes, peak_resident_bytes; /* arena bytes held by admitted requests */
    int64_t resident_sites, peak_resident_sites;
    int32_t active, peak_active; /* resident simulations */
    int64_t launches;          /* kernels launched by this server */
} lbfd_server_stats;

typedef struct lbfd_server *lbfd_server_t;

/* Defaults: FP32, local Gaussian noise, current device, 1 GiB budget, no
 * site limit, 1024 slots, 4 steps ahead, 1 pass, FIFO, occupancy 0, one
 * block per tile (LBFD_WALK_PER_TILE), vx_max 2, solo_sites 2^17. */
int lbfd_server_options_init(lbfd_server_options *opt);

/* Creates a server: one device arena of hbm_budget bytes, two streams
 * (compute and copy), and pinned staging for its tables.  LBFD_ENOMEM if
 * the arena cannot be allocated. */
int lbfd_server_create(lbfd_server_t *out, const lbfd_server_options *opt);

/* Waits for all queued GPU work, then frees everything the server
 * allocated.  Results already copied stay valid; unfinished requests are
 * dropped.  NULL is accepted. */
int lbfd_server_destroy(lbfd_server_t s);

/* Queues a request and returns its id (0, 1, 2, ... in submission order).
 * Touches no GPU state.  LBFD_EINVAL for a malformed request (including
 * Q * sites >= 2^32) and for one
 * that could never be admitted (its blocks exceed the whole budget or the
 * site limit, or no result buffer is given for a result kind that needs
 * one).  in_host and out_host must stay valid until the request is done. */
int lbfd_server_submit(lbfd_server_t s, const lbfd_request *req, int64_t *id);

/* Does up to max_steps rounds of: note finished copies, admit queued
 * requests, launch one time step of every resident simulation.  Returns
 * early when nothing is resident.  Blocks only while max_ahead steps are
 * already queued on the GPU.  *unfinished (may be NULL) = requests not done. */
int lbfd_server_pump(lbfd_server_t s, int32_t max_steps, int64_t *unfinished);

/* Pumps until every submitted request is done. */
int lbfd_server_drain(lbfd_server_t s);

/* State of request id; latency_s (may be NULL) = seconds from submission
 * (or trace arrival) until the host saw its result copy finish, once done. */
int lbfd_server_poll(lbfd_server_t s, int64_t id, int32_t *state, double *latency_s);

int lbfd_server_get_stats(lbfd_server_t s, lbfd_server_stats *st);

/* The request loop for a fixed trace: submits reqs[k] when arrival_s[k]
 * seconds (non-decreasing) have passed since the call began, pumps one
 * step at a time, and returns when all are done.  Results of requests with
 * out_host == NULL go to the caller's pinned buffer sink_host (sink_bytes),
 * in a range reserved when the result is ready (while the sink is full, a
 * finished simulation waits in device memory) and released when its copy is
 * seen done (the contents are not kept).  latency_s[k] = completion - arrival;
 * *makespan_s = last completion - call start.  Requests already submitted
 * are served along with the trace. */
int lbfd_server_run_trace(lbfd_server_t s, const lbfd_request *reqs, const double *arrival_s, int32_t n,
                          void *sink_host, int64_t sink_bytes, double *latency_s, double *makespan_s);

/* ---- host range allocator --------------------------------------------------
 * The first-fit allocator the server carves its device arena and its host
 * result staging with: ranges of [0, capacity), sizes rounded up to
 * `align` (a power of two), freed neighbours coalesced.  Host only. */
typedef struct lbfd_pool *lbfd_pool_t;
int lbfd_pool_create(lbfd_pool_t *out, int64_t capacity, int64_t align);
int lbfd_pool_destroy(lbfd_pool_t p);
/* *offset of a free range of size bytes; LBFD_EBUSY (and *offset = -1) when none fits. */
int lbfd_pool_alloc(lbfd_pool_t p, int64_t size, int64_t *offset);
/* LBFD_EINVAL when no allocated range starts at offset. */
int lbfd_pool_free(lbfd_pool_t p, int64_t offset);
int lbfd_pool_stats(lbfd_pool_t p, int64_t *used, int64_t *largest_free, int32_t *free_ranges);

/* Message for the calling thread's last failure ("" if none). */
const char *lbfd_last_error(void);

/* Number of step-kernel launches the calling process has issued. */
int64_t lbfd_kernel_launches(void);

/* sizeof(lbfd_options), sizeof(lbfd_obs) and sizeof(lbfd_member) as compiled
 * into the library, for bindings that mirror the structs.  Any pointer may be
 * NULL. */
int lbfd_struct_sizes(int64_t *options_bytes, int64_t *obs_bytes, int64_t *member_bytes);

/* sizeof(lbfd_server_options), sizeof(lbfd_request), sizeof(lbfd_server_stats). */
int lbfd_server_struct_sizes(int64_t *options_bytes, int64_t *request_bytes, int64_t *stats_bytes);

#ifdef __cplusplus
}
#endif
#endif /* LBFD_H */
