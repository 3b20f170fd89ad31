// Internal declarations of libnep (GB300 / sm_103a). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace nep {

constexpr int kMaxTypes = 8;
constexpr int kListBuf = 512;   // largest neighbour-list capacity per atom
constexpr int kMaxImage = 3;    // largest cell/image offset searched per axis
// Distance (A) added to r_c^R + skin before a cell is left out of the neighbour search: far
// above the FP32 rounding of a pair distance, so no candidate that the distance test would
// accept is left out.
constexpr double kReachMargin = 2e-3;
constexpr int kAtomBlock = 128; // threads per block of the per-atom kernel
constexpr int kGatherBlock = 128;
constexpr int kReduceSlots = 16; // per-block partial sums: U, KE, W[9], force error, J[3], spare

// Geometry of one neighbour build: the cell grid, the packing of list entries and the
// table of pair shift vectors indexed by the packed image code.
struct Grid {
  int nc[3];          // cells per axis
  int R[3];           // cell offsets searched per axis (1 for large cells)
  int ncell;
  int jbits;          // bits of the atom index in a list entry
  unsigned jmask;
  int obits;          // bits of one offset component in the code (2 or 3)
  int ncode;          // entries of the shift table (2^(3 obits))
  double H[3][3];     // cell rows
  double Hinv[3][3];  // s = r . Hinv
  double Hc[3][3];    // rows of one grid cell: H[a] / nc[a]
  float reach[3];     // (r_c^R + skin + kReachMargin) / cell thickness per axis: a cell whose
                      // gap to an atom's cell position exceeds it along any axis holds no pair
  int cell_off;       // first global cell of this structure (batches; 0 for one structure)
  int dtab_off;       // first shift-table entry of this structure (batches; 0 for one structure)
};

// Structures of a batch: grid of every structure and the structure of every atom (internal
// order). A single structure uses grids == nullptr and the grid passed by value.
struct Batch {
  const Grid *grids;
  const int *sid;
  int n;
  // serving engine: per-structure build requests of the drift kernel. A build that is not
  // forced (BuildStatus::full == 0) then re-sorts and re-lists only the flagged structures;
  // every other structure keeps its atom order, cells, lists and reference positions.
  int *sflag = nullptr;
};

// Per-atom device arrays. Internally atoms are kept in cell order (re-sorted at every
// neighbour rebuild); perm[i] is the caller's index of internal atom i.
struct AtomState {
  double *x, *v, *F, *x_ref, *origin;  // [N][3]
  int *types, *perm, *cell_of;         // [N]
  float4 *pos4;                        // [N] cell-local FP32 coordinates + type bits
  float4 *posA;                        // [N] FP32 coordinates in the structure's cell frame at the
                                       // last build (neighbour search only) + type bits
  double *x2, *v2, *F2;                // reorder scratch [N][3]
  int *types2, *perm2, *cell2;         // reorder scratch [N]
};

// Cell list and neighbour lists.
struct ListBufs {
  int *cell_count, *cell_cursor, *cell_start, *cell_atoms;
  unsigned *nl_r;  // [cap_r][N]
  int *nn_r;       // [T][N]
  unsigned *nl_a;  // [cap_a][N]
  int *nn_a;       // [N]
  int *rev_a;      // [cap_a][N]
  int cap_r, cap_a;
  unsigned *stage_e;        // [cap_r][N] accepted candidates of one build, or null (second scan)
  unsigned char *stage_g;   // [cap_r][N] their groups
};

// Device-visible status written by the builders.
struct BuildStatus {
  int overflow;        // any atom exceeded a list capacity
  int max_r, max_a;    // largest radial/angular list length
  int rev_missing;     // angular pairs without their reverse pair (must stay 0)
  unsigned long long sum_r, sum_a;  // total list entries
  unsigned long long in_r, in_a;    // entries with r < r_c (at build time)
  int rebuild;         // a rebuild is pending (set by the drift kernel or the host)
  int full;            // the pending build covers every structure (forced); else, with
                       // per-structure flags, only the flagged ones
  int bad_input;       // bit 0: type out of range, bit 1: non-finite position
  int tc_timeout;      // a tensor-core completion wait ran out (results invalid)
  long long n_rebuilds;
  long long md_steps;
};

// FIRE minimisation state (Bitzek et al., Phys. Rev. Lett. 97, 170201 (2006)), kept on the
// device so that a relaxation step needs no host round trip.
struct FireState {
  double dt;         // current time step (fs)
  double alpha;      // current mixing factor
  double dt_max;     // largest time step
  double fmax2;      // convergence threshold on max_i |F_i|^2
  int n_pos;         // consecutive steps with P = F . v > 0
  int converged;     // set once max_i |F_i| < fmax: later steps change nothing
  int steps;         // steps taken before convergence
  int pad;
};

// One job of the batched serving engine (a structure of the batch), device resident.
enum { kJobSingle = 0, kJobFire = 1, kJobNve = 2 };
struct EngineSlot {
  int kind;          // kJob*
  int phase;         // 0: initial evaluation this iteration, 1: stepping, 2: finished (frozen)
  int steps_done;    // velocity-Verlet steps taken
  int n_steps;       // NVE: steps to take; FIRE: most steps
  double dt;         // NVE time step (fs)
  FireState fire;    // FIRE state (kind == kJobFire)
};

// A job entering the batched serving engine (host arrays stay valid during engine_relayout).
struct EngineJob {
  int kind, n, n_steps;
  double box[9];
  double dt, fmax;
  const double *pos, *vel;
  const int *types;
};

// Bussi-Donadio-Parrinello velocity rescaling (J. Chem. Phys. 126, 014101 (2007)), device
// resident: the caller's random numbers for every step (R1 ~ N(0,1), S ~ chi^2 with N_f - 1
// degrees of freedom) and the factor of the current step.
struct ThermoState {
  double c;              // exp(-dt / tau)
  double kbar;           // target kinetic energy N_f k_B T0 / 2 (eV)
  double nf;             // degrees of freedom N_f = 3N - 3
  double alpha;          // velocity factor of the last step
  const double *rand;    // [n_steps][2] (R1, S)
  long long step;        // steps thermostatted in this run
};

// Pair vector d = r_j - r_i from cell-local FP32 coordinates and the shift of the image
// code. The explicitly rounded operations make d_ji the exact negation of d_ij, so both
// atoms of a pair take the same inclusion decision in every kernel.
__device__ __forceinline__ float3 pair_vector(const float4 &pi, const float4 &pj, const float4 &D) {
  return make_float3(__fadd_rn(__fsub_rn(pj.x, pi.x), D.x), __fadd_rn(__fsub_rn(pj.y, pi.y), D.y),
                     __fadd_rn(__fsub_rn(pj.z, pi.z), D.z));
}
__device__ __forceinline__ float norm2(const float3 &d) {
  return __fmaf_rn(d.z, d.z, __fmaf_rn(d.y, d.y, __fmul_rn(d.x, d.x)));
}
// pos4.w holds the atom type in bits 0-7 and its structure (batches) in bits 8-31.
__device__ __forceinline__ int type_of(const float4 &p) { return __float_as_int(p.w) & 0xFF; }
__device__ __forceinline__ int struct_of(const float4 &p) { return __float_as_int(p.w) >> 8; }

// Arguments of the per-atom and gather kernels (everything except the model weights).
struct AtomArgs {
  int N, T;
  int jbits;
  unsigned jmask;
  int ncode;
  float rcR, rcA;
  const float4 *pos4;      // [N] cell-local xyz + type bits
  const float4 *dtab;      // [ncode] pair shift vectors
  const unsigned *nl_r;    // [cap_r][N] packed entries, grouped by neighbour type
  const int *nn_r;         // [T][N] radial entries per neighbour type
  const unsigned *nl_a;    // [cap_a][N]
  const int *nn_a;         // [N]
  const int *rev_a;        // [cap_a][N] flat index of the reverse angular pair
  int cap_r, cap_a;        // list capacities (slots per atom), bounds of the list prefetches
  const float *c_r;        // [T][T][nR+1][KR+1] FP32 copy
  const float *c_a;        // [T][T][nA+1][KA+1]
  float *e_rad;            // [N][T][est] radial force coefficients
  int est;
  float4 *p_ang;           // [cap_a][N] angular partial forces
  const int *perm;         // [N] caller index of each internal atom (outputs are scattered)
  double *energy;          // [N] or null
  double *q_out;           // [N][N_des] descriptor output (descriptor mode) or null
  double *partial_atom;    // [gridDim] block sums of U
  // gather outputs
  double *force;           // [N][3] or null (md keeps FP64 forces here)
  double *virial;          // [N][9] or null
  double *partial_gather;  // [gridDim][kReduceSlots]
  // md kick in the gather epilogue
  int md_kick;
  double half_dt;          // dt/2 in fs
  const double *inv_mass_kappa;  // [T] 1 / (m * 103.64...) for a = F * that
  const double *mass_kappa_half; // [T] m * 103.64... / 2 for kinetic energy
  double *vel;             // [N][3]
  // tensor-core network (precision 1): W0 operand tiles in the UMMA layout, error flag
  int precision;           // 0: FP32 network on the FMA pipes; 1: BF16 tensor-core network
  const uint4 *tc_b1;      // GEMM1 operand W0 [NP1 x KP1] (bf16)
  const uint4 *tc_b2;      // GEMM2 operand W0^T [NP2 x KP2] (bf16)
  int *tc_err;             // set when a tensor-core wait ran out
  // Batched kernels only. dtab then holds ncode shift vectors per structure (the structure
  // index sits in pos4.w above the type bits), and blockIdx.y selects the member of a
  // population whose coefficients and network the block uses; every per-member array is
  // offset by member x its stride (in elements).
  const float *pop_ann;    // [P][H*N_des + 2H + 1]: w0, b0, w1, b1 per member, or null
  const uint4 *pop_tc;     // [P][2 tiles] BF16 operand tiles per member (precision 1), or null
  long long s_cr, s_ca, s_ann, s_tc;  // strides of c_r, c_a, pop_ann, pop_tc
  long long s_erad, s_pang;           // strides of e_rad, p_ang
  long long s_out;                    // atoms per member in energy (x1), force (x3), virial (x9)
  const double *f_tar;     // [N][3] caller order, or null: sum of (F_i - F_tar,i)^2 per block
  const FireState *fire;   // FIRE relaxation: kick with its dt, none once converged (or null)
  // heat current J_i = W_i . v_i (Eq. Ji) with the velocities after the kick (MD) or these
  // caller-order velocities; per-atom values in caller order, or null
  const double *vel_in;    // [N][3] caller order, or null
  double *heat;            // [N][3] caller order, or null
  // batched serving engine: per-structure kick (phase, time step, FIRE state), or null
  const EngineSlot *slots;
  // model shape at run time and the FP32 network [w0 | b0 | w1 | b1] on the device: read only
  // by the kernels that take the shape at run time (shapes without a compiled instantiation)
  int gR, gKR, gA, gKA, gH, gL3, gL4, gL5, gD;
  const float *ann;
  // FP32 per-atom kernel form: 1 the register-resident form, 3 the low-register form (three
  // blocks per SM; shapes whose S_nk fit 128 TMEM columns)
  int atom_occ;
};

// Model constants of one handle, FP32.
struct ModelF {
  float c3b[24];
  float c4b[5];
  float c5b[3];
};

// Per-shape launchers (one instantiation per compiled hyper-parameter shape).
struct ShapeOps {
  int nR, KR, nA, KA, H, L3, L4, L5;
  int n_des;
  int kp1, np1;  // tensor-core network tile shapes (K of GEMM1, N of GEMM1)
  cudaError_t (*atom)(const AtomArgs &, const ModelF &, const float *w0, const float *b0, const float *w1,
                      float b1, int descriptor_only, cudaStream_t s);
  cudaError_t (*gather)(const AtomArgs &, cudaStream_t s);
  // batched kernels (per-structure shift tables; `members` population members along y;
  // `block` atoms per CTA: 64 or 128 for the atom kernel (128 with the tensor-core network),
  // 64, 128 or 256 for the gather kernel)
  cudaError_t (*atom_batch)(const AtomArgs &, const ModelF &, const float *w0, const float *b0, const float *w1,
                            float b1, int members, int block, cudaStream_t s);
  cudaError_t (*gather_batch)(const AtomArgs &, int members, int block, cudaStream_t s);
  int (*atom_blocks)(int N);
  int (*gather_blocks)(int N);
  int lowreg;  // the shape's S_nk fit 128 TMEM columns: the low-register FP32 form (3) exists
};

int shape_count();
const ShapeOps *shape_at(int i);
// kernels that take the model shape at run time (any shape within these limits)
constexpr int kGenMaxN = 19;     // n_max^R, n_max^A, N_bas^R, N_bas^A
constexpr int kGenMaxNeu = 256;  // N_neu
constexpr int kGenMaxDes = (kGenMaxN + 1) * 7;
const ShapeOps *shape_generic();

// Host helpers shared by the handle-based and the static-scratch entry points.
struct Grid;
void model_constants(ModelF &m);
int build_grid(const double *box, double rl, int N, Grid &g, float4 *dtab, double *volume, const char **err);
cudaError_t launch_rebuild(int N, int T, const Grid &g, const Batch &B, const float4 *dtab, float rlR2, float rlA2,
                           float rcR2, float rcA2, const AtomState &a, const ListBufs &L, int count_only,
                           BuildStatus *st, cudaStream_t s);
void launch_iota(int N, int *perm, cudaStream_t s);
void launch_export(int N, const AtomState &a, const Grid &g, const Batch &B, double *pos, double *vel, double *force,
                   cudaStream_t s);
void launch_export_lists(int N, int T, const float4 *pos4, const int *perm, const ListBufs &L, const float4 *dtab,
                         int ncode, int jbits, unsigned jmask, int cap, int *nn_r, int *j_r, float *d_r,
                         int *nn_a, int *j_a, float *d_a, cudaStream_t s);
// batches: structure index of every atom, the shift tables of all structures, and the
// per-structure sums of per-atom energies and virials (caller order, per member)
void launch_struct_ids(int n_struct, const int *offsets, int *sid, cudaStream_t s);
void launch_shift_tables(int n_struct, const Grid *grids, int ncode, int obits, float4 *dtab, cudaStream_t s);
// max_atoms: the largest structure (structures above kWideSum atoms are summed by a block)
void launch_struct_sums(int n_struct, int members, const int *offsets, int N, const double *e_atom,
                        const double *w_atom, double *e_struct, double *w_struct, int max_atoms, cudaStream_t s);
void launch_arm_rebuild(BuildStatus *st, cudaStream_t s);
void launch_fire_mix(int N, const AtomState &a, FireState *fire, int check_only, cudaStream_t s);
// batched serving engine
void launch_engine_drift(int N, const AtomState &a, const int *sid, const EngineSlot *slots,
                         const double *inv_mass_kappa, double half_skin2, int *sflag, BuildStatus *st,
                         cudaStream_t s);
void launch_clear_flags(BuildStatus *st, cudaStream_t s);
void launch_engine_fire(int n_struct, const int *offsets, const AtomState &a, EngineSlot *slots, cudaStream_t s);
void launch_engine_advance(int n_struct, EngineSlot *slots, cudaStream_t s);
void launch_engine_relayout(int n_keep, const int4 *table, const AtomState &src, AtomState dst, cudaStream_t s);
void launch_thermostat(int N, const AtomState &a, int nb_gather, const double *partial_gather, ThermoState *ts,
                       cudaStream_t s);
// population evaluation: parameter vectors into kernel arrays, BF16 tiles, Eq. loss
void launch_unpack_population(int n_pop, const double *z, int n_par, int n_cr, int n_ca, float *cr, float *ca,
                              float *ann, double *reg, cudaStream_t s);
void launch_population_tiles(int n_pop, const float *ann, int n_ann, int H, int D, int KP1, int NP1,
                             unsigned short *tiles, cudaStream_t s);
void launch_population_loss(int members, int n_struct, const int *offsets, const double *e_struct,
                            const double *w_struct, const double *e_tar, const double *w_tar,
                            const double *partial_gather, int nb_gather, int N, const double *reg, int n_par,
                            const double *lambda, double *loss, cudaStream_t s);

}  // namespace nep

// Batched serving engine on a library handle (implemented with the C ABI, used by the server).
struct nep_handle;
namespace nep {
int engine_relayout(nep_handle *h, const std::vector<int> &keep, const std::vector<EngineJob> &add, cudaStream_t s,
                    size_t target_bytes = 0);
int engine_step(nep_handle *h, cudaStream_t s, int n_iter, bool force_rebuild);
// neighbour builds of the engine's batch so far (read with the status after every chunk)
long long engine_builds(const nep_handle *h);
int engine_fetch(nep_handle *h, int k, double *pos, double *force, double *vel, cudaStream_t s);
int engine_jobs(const nep_handle *h);
int engine_atoms(const nep_handle *h);
const EngineSlot &engine_slot(const nep_handle *h, int k);
double engine_energy(const nep_handle *h, int k);
const double *engine_virial(const nep_handle *h, int k);
void set_thread_alloc_stream(cudaStream_t s);
void release_workspace(nep_handle *h);
size_t workspace_bytes(nep_handle *h);
cudaError_t stream_sync(cudaStream_t s);
}  // namespace nep
