/*
 * libnep: GB300 (sm_103a) evaluation of the NEP3 machine-learned potential of
 * arXiv:2205.10046 (energy, forces, virials) and a velocity-Verlet NVE driver.
 *
 * What the library computes (all of it in its own CUDA kernels):
 *   - cell-list neighbour search into a radial list (r < r_c^R + skin) and an angular
 *     list (r < r_c^A + skin), all periodic images included (the quantities NN_i^R,
 *     NN_i^A, NL_im^R, NL_im^A listed at the start of Appendix B);
 *   - the radial descriptor of Eq. qin with the Chebyshev radial functions of Eqs. g_n
 *     and f_n and per-ordered-type-pair coefficients c_nk^{t_i t_j} (Sec. II B);
 *   - the angular sums S_{n,k} of Eq. S_nk and the 3-body (q_nl, l <= 4), 4-body (q_n222)
 *     and 5-body (q_n1111) components with the pre-computed coefficients of Sec. II D;
 *   - the single-hidden-layer tanh network of Eq. Ui and its gradient dU_i/dq;
 *   - the partial forces of Eq. partial_force, gathered into F_i (Eqs. F_ij, F_i) and
 *     the per-atom virial W_i (Eq. virial) without atomics;
 *   - a velocity-Verlet NVE step (the NVE ensemble named in Sec. III A).
 *
 * Units: Angstrom, fs, eV, atomic mass unit, K.
 * Conventions:
 *   positions  [N][3] FP64, any values (they are wrapped into the cell internally);
 *   cell       `box` [3][3] FP64, ROWS are the cell vectors a, b, c; r = s . box for
 *              fractional s; any right- or left-handed non-degenerate cell;
 *   types      [N] int32 in [0, n_types);
 *   forces     [N][3] FP64;
 *   virials    [N][9] FP64 in the order xx, yy, zz, xy, xz, yz, yx, zx, zy with
 *              W_i[a][b] = sum_j (r_j - r_i)_a (dU_j/dr_ji)_b (Eq. virial); the total
 *              is -(dE/d eps)^T for an affine strain r -> (I + eps) r;
 *   energies   per-atom site energies U_i and their FP64 sum.
 * Arithmetic: pair vectors, descriptors, network and partial forces in FP32; positions,
 * velocities, integration and the energy/virial totals in FP64 (the mixed precision
 * of Sec. II G: FP64 inputs/outputs, FP32 internals).
 *
 * Descriptor layout (the paper fixes the components, not their order):
 *   q = [ q_n (n = 0..n_R) | q_n1 (n = 0..n_A) | q_n2 | q_n3 | q_n4 | q_n222 | q_n1111 ].
 *
 * Errors: every call returns NEP_OK (0) or a negative NEP_ERR_* code; nothing throws
 * across the ABI. nep_last_error() gives a message for the last failed call on a handle.
 * A handle is not thread-safe: serialise calls that share one.
 */
#ifndef NEP_H
#define NEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEP_OK 0
#define NEP_ERR_ARG (-1)               /* invalid argument (null pointer, bad size, bad type) */
#define NEP_ERR_OOM (-2)               /* device allocation failed */
#define NEP_ERR_CUDA (-3)              /* a CUDA runtime call failed */
#define NEP_ERR_NEIGHBOR_OVERFLOW (-4) /* an atom has more neighbours than the list can hold */
#define NEP_ERR_NONFINITE (-5)         /* non-finite position, force or energy */
#define NEP_ERR_UNSUPPORTED (-6)       /* hyper-parameters without a compiled kernel, or a cell
                                          thinner than a third of the list radius */
#define NEP_ERR_STATE (-7)             /* call out of order (e.g. md_run before md_init) */
#define NEP_ERR_TIMEOUT (-8)           /* a device-side wait ran out (tensor-core completion) */

#define NEP_MAX_TYPES 8

/* Opaque library state: model, device workspace, neighbour lists, MD state. */
typedef struct nep_handle nep_handle;

/* Stream type without pulling in the CUDA headers: pass a cudaStream_t (0 = legacy
 * default stream). */
typedef void *nep_stream_t;

/* Model hyper-parameters and weights (the nep.in keywords of Sec. III A plus the
 * trained parameters). All pointers are HOST pointers; nep_create copies everything,
 * the caller keeps ownership. */
typedef struct {
  int version;          /* must be 3 (NEP3) */
  int n_types;          /* 1..NEP_MAX_TYPES */
  double rc_radial;     /* r_c^R > 0 (Angstrom) */
  double rc_angular;    /* 0 < r_c^A <= r_c^R */
  int n_max_radial;     /* n_max^R >= 0 */
  int n_max_angular;    /* n_max^A >= 0 */
  int basis_radial;     /* N_bas^R >= 0 (K_R + 1 Chebyshev functions) */
  int basis_angular;    /* N_bas^A >= 0 */
  int l_max_3b;         /* 1..4 */
  int l_max_4b;         /* 0 (off) or 2 (q_n222; l = 1 and l = 3 vanish, Sec. II D) */
  int l_max_5b;         /* 0 (off) or 1 (q_n1111) */
  int n_neuron;         /* N_neu >= 1 */
  const double *c_radial;  /* [T][T][n_max_radial+1][basis_radial+1], ordered (t_i, t_j) */
  const double *c_angular; /* [T][T][n_max_angular+1][basis_angular+1] */
  const double *w0;        /* [n_neuron][N_des], neuron-major (w^(0)_{mu nu} of Eq. Ui) */
  const double *b0;        /* [n_neuron] */
  const double *w1;        /* [n_neuron] */
  double b1;
  const double *mass;      /* [T] in u; needed by md_* only (may be NULL otherwise) */
  double skin;             /* neighbour-list skin in Angstrom; <= 0 selects 1.0 */
} nep_params;

/* Create a handle for one model. Validates the parameters (NEP_ERR_ARG) and checks that
 * a kernel is compiled for (n_max^R, N_bas^R, n_max^A, N_bas^A, N_neu, l_max's)
 * (NEP_ERR_UNSUPPORTED otherwise; nep_supported() lists them). Allocates nothing on
 * the device until the first compute or md_init. Uses the current CUDA device. */
int nep_create(const nep_params *params, nep_handle **out);

/* Release the handle and all device memory it owns. NULL is accepted. */
int nep_destroy(nep_handle *h);

/* Message for the last failed call on h (or for the last failed nep_create when h is NULL).
 * Valid until the next call on the handle. */
const char *nep_last_error(const nep_handle *h);

/* One NEP3 evaluation (Sec. II; the four-kernel scheme of Sec. II G / Appendix B,
 * re-organised for GB300: neighbour build, one fused per-atom kernel for descriptor,
 * network and angular partial forces, one gather kernel for F and W).
 * DEVICE pointers, stream-ordered on `stream`: pos [N][3], types [N]; outputs
 * energy [N] (or NULL), energy_total [1] (or NULL), force [N][3] (required),
 * virial [N][9] (or NULL), virial_total [9] (or NULL). `box` is a HOST pointer [3][3].
 * The neighbour lists are rebuilt on every call. The call synchronises `stream` once
 * (to size the neighbour lists) and returns with the kernels queued on `stream`.
 * n_atoms == 0 is valid and writes zero totals. The library owns its workspace. */
int nep_compute(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                double *energy, double *energy_total, double *force, double *virial,
                double *virial_total, nep_stream_t stream);

/* nep_compute with HOST pointers for every array (synchronous; copies in and out). */
int nep_compute_host(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                     double *energy, double *energy_total, double *force, double *virial,
                     double *virial_total);

/* Many independent periodic structures in one evaluation (batched form of nep_compute; the
 * training set of Sec. III is such a batch, evaluated for every candidate of Eq. loss).
 * Structure s owns atoms [offsets[s], offsets[s+1]) of the concatenated arrays and the cell
 * rows boxes[s][3][3]; thin cells are handled with all their periodic images (up to 3 cell
 * lengths per axis: an image range above that returns NEP_ERR_UNSUPPORTED naming the
 * structure). offsets [n_struct+1] (offsets[0] = 0, non-decreasing) and boxes [n_struct][9]
 * are HOST pointers; the rest are DEVICE pointers, N = offsets[n_struct]: pos [N][3],
 * types [N]; outputs energy [N] (or NULL), energy_struct [n_struct] (or NULL: E_s = sum of
 * U_i over the structure), force [N][3] (required), virial [N][9] (or NULL), virial_struct
 * [n_struct][9] (or NULL: sum of W_i). Empty structures are allowed (zero sums). The grids of
 * the last layout (offsets and boxes) are kept and reused while it repeats. Synchronises
 * `stream` to size the neighbour lists, like nep_compute; errors as nep_compute. */
int nep_compute_batch(nep_handle *h, int n_struct, const int *offsets, const double *pos, const int *types,
                      const double *boxes, double *energy, double *energy_struct, double *force,
                      double *virial, double *virial_struct, nep_stream_t stream);

/* Number of trainable parameters N_par of the handle's model (Sec. II E): the length of one
 * candidate vector z of nep_eval_population, ordered c^R [T][T][n_R+1][K_R+1],
 * c^A [T][T][n_A+1][K_A+1], w0 [N_neu][N_des], b0 [N_neu], w1 [N_neu], b1. */
int nep_n_par(const nep_handle *h);

/* Loss of Eq. loss for a population of candidate parameter vectors on one structure set,
 * the inner step of the evolutionary training of Sec. III. Every candidate gets its own
 * descriptor coefficients and network; the hyper-parameters (cut-offs, basis sizes, types)
 * are the handle's, its own weights are not used.
 *   z       DEVICE [n_pop][N_par] FP64 candidate vectors (order of nep_n_par)
 *   offsets HOST [n_struct+1], boxes HOST [n_struct][9], pos DEVICE [N][3], types DEVICE [N]:
 *           the structure set, as nep_compute_batch (N = offsets[n_struct] > 0)
 *   e_tar   DEVICE [n_struct] target energy per atom (eV/atom; empty structures ignored)
 *   f_tar   DEVICE [N][3] target forces (eV/Angstrom)
 *   w_tar   DEVICE [n_struct][6] target virial per atom (eV/atom; xx, yy, zz, xy, yz, zx,
 *           compared with the symmetric part of W_s / N_s), or NULL (no virial term)
 *   lambda  HOST [5]: lambda_e, lambda_f, lambda_v, lambda_1, lambda_2
 *   loss    DEVICE [n_pop][6] out: L, RMSE_E, RMSE_F, RMSE_W, sum|z|/N_par, sqrt(sum z^2/N_par)
 * Members are evaluated several per launch (grid.y; nep_set_tuning), in FP32 (or with the
 * BF16 tensor-core network after nep_set_precision(h, 1)); every sum is FP64 in a fixed
 * order, so the losses do not depend on the grouping. Synchronises `stream` once (list
 * sizing); errors as nep_compute_batch. */
int nep_eval_population(nep_handle *h, int n_pop, const double *z, int n_struct, const int *offsets,
                        const double *pos, const int *types, const double *boxes, const double *e_tar,
                        const double *f_tar, const double *w_tar, const double *lambda, double *loss,
                        nep_stream_t stream);

/* Launch shapes of the batched kernels (nep_compute_batch, nep_eval_population). Zero
 * fields select the defaults. The shapes change the speed, not the per-atom results. */
typedef struct {
  int members_per_launch; /* population members per launch (grid.y); 0: as many as a workspace
                             budget of min(half the free memory, 32 GiB) holds */
  int atom_block;         /* atoms per CTA of the batched per-atom kernel: 64 or 128 (0: 128;
                             the BF16 tensor-core network always uses 128-atom tiles) */
  int gather_block;       /* atoms per CTA of the batched gather kernel: 64, 128, 256 (0: 128) */
  int last_members;       /* out: members per launch used by the last nep_eval_population */
  int n_tried;            /* out: candidates timed by the last nep_autotune */
  float best_ms;          /* out: time of one evaluation (per member) with the chosen shapes */
  float default_ms;       /* out: the same with 128 / 128 atoms per CTA and one member */
  int atom_form;          /* per-atom kernel form (FP32 and BF16 networks): 1 = sums and
                             dU/dS_nk in registers (two CTAs per SM), 3 = two passes for S_nk and
                             dU/dS_nk in shared memory (three CTAs per SM; shapes whose
                             (n_max^A + 1) x 24 sums fit 128 TMEM columns, else as 1; with the
                             BF16 networks (precision 1 and 2) S_nk waits in shared memory and
                             the GEMM operands and results use 128 TMEM columns); 0 = the
                             library's default (3 where it exists). nep_get_tuning returns the
                             form in use. The form applies to
                             128-atom CTAs (an atom_block of 64 runs form 1) and nep_autotune keeps
                             it. The two forms agree to FP32 rounding; within one form, results do
                             not depend on the CTA sizes. */
} nep_tuning;

/* Set or read the launch shapes (NEP_ERR_ARG for values outside the lists above). */
int nep_set_tuning(nep_handle *h, const nep_tuning *t);
int nep_get_tuning(const nep_handle *h, nep_tuning *t);

/* Autotuner: builds the neighbour lists of the structure set (arguments as
 * nep_compute_batch), times the atom and gather kernels for every atoms-per-CTA pair (best of
 * three launches after a warm-up, CUDA events on `stream`) and, when n_pop > 0, members per
 * launch 1, 2, 4, ... up to n_pop (or the workspace budget) with the best pair; keeps the
 * fastest shapes in the handle and returns them in *out (may be NULL). Synchronous. */
int nep_autotune(nep_handle *h, int n_struct, const int *offsets, const double *pos, const int *types,
                 const double *boxes, int n_pop, nep_tuning *out, nep_stream_t stream);

/* ------------------------------------------------------------------------ serving
 * A persistent request loop with iteration-level (continuous) batching; the paper has no
 * counterpart. Jobs on structures of any size are queued; a scheduler thread keeps every
 * running job as one structure of a device-resident batch and advances all of them by one
 * iteration at a time (one velocity-Verlet or FIRE step each, or a job's first evaluation),
 * with the batched kernels of nep_compute_batch. Between iterations finished jobs leave and
 * queued jobs join, first in first out, while the batch has a free job slot and the jobs'
 * workspace estimates fit the memory budget; positions, velocities and lists stay on the
 * device. Neighbour lists (radius r_c + the params' skin) are rebuilt after every change of
 * the batch and whenever an atom has moved more than skin/2. A job's arithmetic uses only its
 * own structure, so its results do not depend on what else runs, up to the order of its pair
 * sums (which follows its last list build): equal alone and in a mix within FP32 rounding. */
#define NEP_JOB_SINGLE 0 /* one energy / force / virial evaluation (nep_compute) */
#define NEP_JOB_FIRE 1   /* FIRE relaxation (fire_run), then one evaluation at the result */
#define NEP_JOB_NVE 2    /* velocity-Verlet NVE (md_run), then one evaluation at the end */

typedef struct nep_server nep_server;

typedef struct {
  size_t memory_budget; /* bytes of device workspace that running jobs may hold together */
  int workers;          /* job slots of the batch: jobs on the device at once (1..65536) */
  int precision;        /* 0: FP32 network, 1: BF16 / 2: split-BF16 tensor-core network (nep_set_precision) */
  int compact_every;    /* 0: a finished job leaves the batch at once (one layout change, with a
                           full neighbour build, per iteration that ends a job); c > 0: finished
                           jobs stay frozen in the batch (results already delivered) until they
                           are 1/c of it, and queued jobs join once 1/c of the slots and of the
                           budget are free, so one layout change serves many jobs */
  int min_chunk;        /* iterations between two reads of the job states (0 or 1: a single
                           iteration whenever a job starts or could join, else up to the first
                           completion); k > 1 runs at least k (at most 32): jobs that finish
                           inside a chunk stay frozen until it ends, which spreads the per-chunk
                           host work (checkpoint, status and state reads) over k iterations */
} nep_server_config;

typedef struct {
  int kind;             /* NEP_JOB_* */
  int n_atoms;          /* >= 1 */
  const double *pos;    /* HOST [N][3]; copied by nep_server_submit */
  const int *types;     /* HOST [N] */
  const double *vel;    /* HOST [N][3] initial velocities for NVE (A/fs), or NULL (zero) */
  double box[9];        /* cell rows */
  int n_steps;          /* FIRE: most steps; NVE: steps */
  double dt_fs;         /* NVE time step; FIRE initial time step */
  double fmax;          /* FIRE convergence threshold on max |F_i| (eV/A) */
} nep_job;

typedef struct {
  long long id;
  int status;           /* NEP_OK or the NEP_ERR_* code of the failed step */
  int kind, n_atoms;
  int steps;            /* MD or FIRE steps taken (FIRE: before convergence) */
  double energy;        /* potential energy of the final state (eV) */
  double virial[9];     /* total virial of the final state (eV) */
  double t_submit, t_start, t_done; /* seconds since nep_server_create: queued, on a worker, done */
  size_t workspace_est; /* device bytes reserved for the job by admission */
  size_t workspace_used;/* device workspace of the whole batch when the job ended */
  char message[160];    /* error text when status != NEP_OK */
} nep_result;

typedef struct {
  int queued, running;
  long long completed, failed;
  size_t bytes_reserved, peak_bytes_reserved; /* admission estimates of the running jobs */
  size_t peak_workspace_bytes;                /* largest device workspace of the batch */
  double atom_evaluations;                    /* sum over finished jobs of N x force evaluations */
  long long iterations, relayouts;            /* batch iterations run; layout changes */
  double relayout_seconds, step_seconds, fetch_seconds; /* scheduler wall time: layout changes,
                                                 iterations (incl. builds and the state read),
                                                 copying finished jobs out */
  long long builds;                           /* neighbour builds of the batch (layout changes
                                                 and skin-triggered rebuilds, overflow replays) */
} nep_server_stats;

/* Start the workers (each creates its handle for `params`, copied). NEP_ERR_ARG for a bad
 * configuration, as nep_create for bad parameters. */
int nep_server_create(const nep_params *params, const nep_server_config *cfg, nep_server **out);
/* Queue a job (HOST arrays copied); *id receives its id. Thread-safe; does not wait for the
 * device. NEP_ERR_OOM if the job alone needs more than the memory budget; NEP_ERR_UNSUPPORTED
 * above 2^23 atoms (a batch holds at most 2^23 atoms in all; admission waits for room). */
int nep_server_submit(nep_server *s, const nep_job *job, long long *id);
/* Next finished job in completion order: waits up to timeout_s seconds (< 0: no limit);
 * NEP_ERR_TIMEOUT if none finished in time. */
int nep_server_wait(nep_server *s, double timeout_s, nep_result *out);
/* Final positions (wrapped into the cell), forces and velocities of a finished job into
 * HOST buffers [N][3] (any may be NULL); the server then drops them. NEP_ERR_ARG for an
 * unknown id or a second call. */
int nep_server_arrays(nep_server *s, long long id, double *pos, double *force, double *vel);
int nep_server_stats_get(nep_server *s, nep_server_stats *out);
/* Finish the jobs on the workers, drop the queued ones, release everything. */
int nep_server_destroy(nep_server *s);

/* Descriptor vectors q^i (Eqs. qin and S_nk with the explicit components of Sec. II D)
 * into q [N][N_des] FP64 (DEVICE pointers, as nep_compute). */
int nep_descriptors(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                    double *q, nep_stream_t stream);

/* Descriptor length N_des of the handle's model (Sec. II D). */
int nep_n_des(const nep_handle *h);

/* Load an MD state (DEVICE pointers): positions [N][3], types [N], velocities [N][3]
 * (Angstrom/fs; NULL = zero) and the HOST cell [3][3]. Builds the neighbour lists and
 * the initial forces. The state then stays on the device. Needs params->mass. */
int md_init(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
            const double *vel, nep_stream_t stream);

/* md_init from HOST arrays (synchronous; the legacy default stream). The arrays are copied
 * straight into the handle's workspace: page-locked host memory gives full-speed copies. */
int md_init_host(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                 const double *vel);

/* Advance n_steps velocity-Verlet NVE steps of dt_fs: v += dt/2 F/m; x += dt v;
 * [neighbour rebuild when an atom moved more than skin/2 since the last build];
 * F = F(x); v += dt/2 F/m. Every `thermo_every` steps (>= 1) one row of `thermo`
 * (DEVICE pointer, or NULL) receives {E_pot, E_kin, T, P} in eV, eV, K, GPa for the
 * state after that step (row r = step (r+1)*thermo_every of this call); thermo must hold
 * n_steps / thermo_every rows of 4 doubles. Each step replays one captured CUDA graph.
 * Returns NEP_ERR_NEIGHBOR_OVERFLOW if a rebuild found more neighbours than the lists
 * hold (the state is then unusable; call md_init again). */
int md_run(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo, nep_stream_t stream);

/* Options of md_run_ex. */
typedef struct {
  int thermo_every;          /* >= 1: rows of thermo and heat_current every thermo_every steps */
  double *thermo;            /* DEVICE [n_steps/thermo_every][4] as md_run, or NULL */
  double *heat_current;      /* DEVICE [n_steps/thermo_every][3]: total heat current J = sum_i W_i . v_i
                                (Eqs. Ji and J-1; eV A/fs) after the step, or NULL */
  double temperature;        /* > 0: Bussi-Donadio-Parrinello thermostat at this temperature (K);
                                <= 0: NVE */
  double tau_fs;             /* thermostat coupling time (fs) */
  const double *bdp_random;  /* DEVICE [n_steps][2]: per step R1 ~ N(0,1) and S ~ chi^2 with 3N-4
                                degrees of freedom, drawn by the caller (thermostat only) */
} md_options;

/* md_run with options: the heat current of Eq. Ji summed over atoms (Eq. J-1) after every
 * thermo row's step, and an NVT thermostat (the paper's MD engine offers several, Sec. III A;
 * this is the Bussi-Donadio-Parrinello one, J. Chem. Phys. 126, 014101 (2007)): after each
 * velocity-Verlet step every velocity is scaled by alpha with
 *   alpha^2 = c + (1 - c)(S + R1^2) Kbar / (N_f K) + 2 R1 sqrt(c (1 - c) Kbar / (N_f K)),
 * c = exp(-dt/tau), N_f = 3N - 3, Kbar = N_f k_B T / 2, K the kinetic energy after the step,
 * and the sign of alpha that of R1 + sqrt(c N_f K / ((1 - c) Kbar)). thermo rows then hold the
 * rescaled kinetic energy and temperature. Errors as md_run. */
int md_run_ex(nep_handle *h, int n_steps, double dt_fs, const md_options *opt, nep_stream_t stream);

/* Per-atom heat current J_i = W_i . v_i (Eq. Ji) of one configuration with the caller's
 * velocities (DEVICE pointers, caller order): heat [N][3] (or NULL) and the total
 * heat_total [3] (or NULL), in eV A/fs. Stream-ordered like nep_compute. */
int nep_heat_current(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                     const double *vel, double *heat, double *heat_total, nep_stream_t stream);

/* FIRE energy minimisation (Bitzek et al., Phys. Rev. Lett. 97, 170201 (2006); the paper
 * has no counterpart) from the state of md_init, with its velocities set to zero. A step is
 * one velocity-Verlet step of the current length dt followed by the FIRE update with
 * P = F . v, |F| and |v| over all atoms: P > 0 mixes v <- (1 - alpha) v + alpha |v| F/|F|
 * and, after more than N_min = 5 such steps in a row, sets dt <- min(1.1 dt, 10 dt0) and
 * alpha <- 0.99 alpha; P <= 0 sets v <- 0, dt <- dt/2, alpha <- alpha_start = 0.1. The
 * relaxation stops (nothing moves again) once max_i |F_i| < fmax, checked on the starting
 * forces and after every step, or after n_steps. thermo: as md_run with thermo_every = 1
 * (n_steps rows; rows after convergence repeat the last state), or NULL. *steps_taken
 * (HOST, or NULL) receives the steps taken before convergence. The state stays resident
 * (md_get_state, md_run). Synchronous; errors as md_run. */
int fire_run(nep_handle *h, int n_steps, double dt0_fs, double fmax, double *thermo, int *steps_taken,
             nep_stream_t stream);

/* md_run without the final synchronisation: queues the n_steps graph replays on `stream`
 * and returns. A neighbour-list overflow during these steps is reported by the next
 * md_status (or md_run) call instead. Same arguments as md_run. */
int md_run_async(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo,
                 nep_stream_t stream);

/* Synchronise `stream` and report the MD health: NEP_OK, or NEP_ERR_NEIGHBOR_OVERFLOW if a
 * rebuild since md_init found more neighbours than the lists hold (the state is then
 * unusable; call md_init again). */
int md_status(nep_handle *h, nep_stream_t stream);

/* Copy the MD state out (DEVICE pointers; any may be NULL): positions wrapped into the
 * cell [N][3], velocities [N][3], forces of the current positions [N][3]. */
int md_get_state(nep_handle *h, double *pos, double *vel, double *force, nep_stream_t stream);

/* md_get_state into HOST arrays (synchronous; the legacy default stream), through the
 * handle's workspace (no temporary device allocation). */
int md_get_state_host(nep_handle *h, double *pos, double *vel, double *force);

/* Statistics of the last neighbour build and of the MD run so far. */
typedef struct {
  int n_atoms;
  int cap_radial, cap_angular;   /* list capacity per atom */
  int max_radial, max_angular;   /* largest list length at the last build */
  double mean_radial, mean_angular;            /* mean list length (r < r_c + skin) */
  double mean_radial_in_rc, mean_angular_in_rc; /* mean count with r < r_c (last build) */
  long long n_rebuilds;          /* neighbour rebuilds since md_init */
  long long md_steps;            /* MD steps since md_init */
  int cells[3];                  /* cell grid */
  int graph_kernels;             /* kernel nodes in the captured MD step graph (0 before md_run) */
  int rebuild_kernels;           /* kernels of one neighbour rebuild (run only on rebuild steps) */
  int batch_graph_kernels;       /* kernel nodes in the captured nep_compute_batch graph (0: none) */
} nep_stats;

int nep_get_stats(nep_handle *h, nep_stats *out);

/* Kernel timing for roofline reports. When enabled, md_run and nep_compute record CUDA
 * events around each library kernel on the launching stream. nep_kernel_times returns,
 * for the most recent call, the device time in ms of each kernel slot (names via
 * nep_kernel_name; slots that did not run report 0). */
int nep_set_profiling(nep_handle *h, int enable);

/* Arithmetic of the network (Eq. Ui) and its gradient dU/dq:
 *   0 (default) FP32 on the FMA pipes;
 *   1 BF16 operands on the tensor cores (tcgen05.mma, FP32 accumulation in tensor memory):
 *     descriptor -> hidden and hidden -> dU/dq as two GEMMs per 128-atom tile. Descriptors,
 *     partial forces and all accumulations stay FP32; integration and totals FP64.
 *     Operand rounding (2^-9 relative) gives forces about 1e-2 relative error.
 *   2 split BF16: as 1, but every operand value x is carried as two BF16 terms
 *     x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and each GEMM adds the three products
 *     hi.hi + lo.hi + hi.lo (the lo.lo term, ~2^-18 relative, is dropped): three times the
 *     tensor-core work, errors near the FP32 form's (about 1e-5 relative).
 * Applies to nep_compute and md_run (nep_descriptors has no network). */
int nep_set_precision(nep_handle *h, int mode);

/* How md_run captures the neighbour rebuild in its step graph: 1 (default) = inside a
 * conditional graph node that runs only when a rebuild is due; 0 = as ordinary kernel
 * nodes that return at once when no rebuild is due (for profilers that cannot look inside
 * graphs with conditional nodes). Results are identical. */
int nep_set_graph_conditional(nep_handle *h, int enable);
int nep_kernel_slots(void);
const char *nep_kernel_name(int slot);
int nep_kernel_times(nep_handle *h, float *ms_out, int n_slots);

/* Descriptor evaluation for callers that cannot allocate device memory (for example a
 * host program whose device memory is planned up front, or code where cudaMalloc must not
 * be called). Same arguments and results as nep_descriptors, but the model is passed
 * directly (no handle, which would allocate) and every scratch array comes from one fixed
 * device array inside the library: NEP_STATIC_SCRATCH_BYTES on every GPU that loads the
 * library, held until the process exits. No cudaMalloc, cudaFree or other allocating call
 * is made.
 *   - n_atoms above NEP_STATIC_MAX_ATOMS, or neighbour lists that do not fit the scratch,
 *     are rejected with NEP_ERR_ARG; nep_last_error(NULL) gives the message.
 *   - The first call on a device looks up the scratch address on that device (with the
 *     device current); make that first call before any stream capture.
 *   - All calls share the one scratch array, which keeps the previous call's contents (each
 *     call rewrites what it reads). Calls that overlap on the GPU race with each other:
 *     serialise them (one stream, or synchronise between calls).
 *   - The call synchronises `stream` twice (to size the neighbour lists) and returns with
 *     the descriptor kernel queued on `stream`.
 *   - Code loading: with CUDA's default lazy module loading the driver loads a kernel's
 *     module, and the arena, the first time they are used, and may allocate device memory
 *     for them then. The first call per hyper-parameter shape on a device can therefore
 *     allocate inside the driver; later calls allocate nothing. A caller that must not
 *     allocate at all makes one warm-up call first, or sets CUDA_MODULE_LOADING=EAGER.
 *   - Per-atom lists longer than 512 entries return NEP_ERR_NEIGHBOR_OVERFLOW, as in the
 *     handle-based calls.
 * The paper has no counterpart: this is a deployment variant of nep_descriptors. */
#define NEP_STATIC_MAX_ATOMS 4096
#define NEP_STATIC_SCRATCH_BYTES (16u << 20)
int nep_descriptors_static(const nep_params *params, int n_atoms, const double *pos, const int *types,
                           const double *box, double *q, nep_stream_t stream);

/* The neighbour lists of the handle's last build, in the caller's atom order: the
 * quantities NN_i^R, NL_im^R, NN_i^A and NL_im^A that the force kernels take as given
 * (Appendix B), with the image of every entry made explicit by its pair vector.
 *   nn_r [N], nn_a [N]        entries of atom i's radial and angular list;
 *   j_r  [N][cap], j_a [N][cap]  caller index j of entry m (m < nn);
 *   d_r  [N][cap][3], d_a [N][cap][3]  FP32 pair vector r_j - r_i (+ the periodic image) of
 *                              entry m, as the kernels form it, at the current positions.
 * Lists hold every pair within r_c + skin (radial) or r_c^A + skin (angular); the radial list
 * is grouped by neighbour type (type 0 first). All outputs are HOST buffers owned by the
 * caller; N is the atom count of the last nep_compute, nep_compute_batch (all structures,
 * concatenated) or md_init/md_run. NEP_ERR_STATE if no lists exist; NEP_ERR_ARG if cap is
 * below the longest list (nep_stats.max_radial / max_angular). Synchronises the device;
 * allocates temporary device memory. For tests and inspection; not on the hot path. */
int nep_export_lists(nep_handle *h, int cap, int *nn_r, int *j_r, float *d_r, int *nn_a, int *j_a, float *d_a);

/* Compiled hyper-parameter shapes: writes up to `max` rows of 8 ints
 * (n_max^R, N_bas^R, n_max^A, N_bas^A, N_neu, l_max^3b, l_max^4b, l_max^5b) and
 * returns the number of shapes. */
int nep_supported(int *shapes, int max);

#ifdef __cplusplus
}
#endif

#endif /* NEP_H */
