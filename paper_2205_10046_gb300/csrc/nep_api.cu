// libnep C ABI (include/nep.h): handle management, validation, device workspace,
// neighbour-list sizing, the compute pipeline and the captured MD step.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nep.h"
#include "nep_internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace nep {
// A named NVTX range around a host call (for timeline profilers; no cost without one).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace nep

namespace nep {
void launch_rebuild_condition(cudaGraphConditionalHandle hc, const BuildStatus *st, cudaStream_t s);
void launch_drift(int N, const AtomState &a, const double *inv_mass_kappa, double dt, double half_skin2,
                  BuildStatus *st, cudaStream_t s, const FireState *fire);
void launch_finalize(int nb_atom, const double *partial_atom, int nb_gather, const double *partial_gather,
                     double *energy_total, double *virial_total, double *heat_total, double *thermo_stage,
                     int *thermo_ctl, int N, double volume, const ThermoState *ts, cudaStream_t s);
constexpr int kThermoCols = 8;  // staged thermo row: E, KE, T, P, J[3], thermostat factor
const ShapeOps *shape_si();
const ShapeOps *shape_pbte();
const ShapeOps *shape_mixed();

int shape_count() { return 3; }
const ShapeOps *shape_at(int i) {
  switch (i) {
    case 0: return shape_si();
    case 1: return shape_pbte();
    case 2: return shape_mixed();
    default: return nullptr;
  }
}
}  // namespace nep

using namespace nep;

namespace nep {

// The paper's 3-body (C3b), 4-body (C4b) and 5-body (C5b) coefficients (Sec. II D),
// evaluated here from the printed expressions.
void model_constants(ModelF &m) {
  const double p = 3.14159265358979323846;
  const double c3[24] = {3.0 / (4 * p), 3.0 / (4 * p), 3.0 / (4 * p),
                         5.0 / (16 * p), 15.0 / (4 * p), 15.0 / (4 * p), 15.0 / (16 * p), 15.0 / (16 * p),
                         7.0 / (16 * p), 21.0 / (32 * p), 21.0 / (32 * p), 105.0 / (16 * p), 105.0 / (16 * p),
                         35.0 / (32 * p), 35.0 / (32 * p),
                         9.0 / (256 * p), 45.0 / (32 * p), 45.0 / (32 * p), 45.0 / (64 * p), 45.0 / (64 * p),
                         315.0 / (32 * p), 315.0 / (32 * p), 315.0 / (256 * p), 315.0 / (256 * p)};
  for (int k = 0; k < 24; ++k) m.c3b[k] = (float)c3[k];
  const double y20 = 0.25 * std::sqrt(5.0 / p), y21 = 0.5 * std::sqrt(7.5 / p), y22 = 0.25 * std::sqrt(7.5 / p);
  m.c4b[0] = (float)(-std::sqrt(2.0 / 35.0) * y20 * y20 * y20);
  m.c4b[1] = (float)(-6.0 * std::sqrt(1.0 / 70.0) * y20 * y21 * y21);
  m.c4b[2] = (float)(6.0 * std::sqrt(2.0 / 35.0) * y20 * y22 * y22);
  m.c4b[3] = (float)(6.0 * std::sqrt(3.0 / 35.0) * y21 * y21 * y22);
  m.c4b[4] = (float)(-12.0 * std::sqrt(3.0 / 35.0) * y21 * y21 * y22);
  m.c5b[0] = (float)(21.0 / (80.0 * p * p));
  m.c5b[1] = (float)(21.0 / (40.0 * p * p));
  m.c5b[2] = (float)(21.0 / (80.0 * p * p));
}

// Cell grid, image range and shift table (dtab[0..ncode), at most 512 entries; skipped when
// dtab is null) for the cell rows `box` and the list radius rl. Returns NEP_OK or an error
// code with *err set.
int build_grid(const double *box, double rl, int N, Grid &g, float4 *dtab, double *volume, const char **err) {
  g.cell_off = 0;
  g.dtab_off = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.H[a][b] = box[3 * a + b];
  double cof[3][3];
  const double(*H)[3] = g.H;
  cof[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
  cof[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
  cof[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
  cof[1][0] = H[2][1] * H[0][2] - H[2][2] * H[0][1];
  cof[1][1] = H[2][2] * H[0][0] - H[2][0] * H[0][2];
  cof[1][2] = H[2][0] * H[0][1] - H[2][1] * H[0][0];
  cof[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
  cof[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
  cof[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];
  const double det = H[0][0] * cof[0][0] + H[0][1] * cof[0][1] + H[0][2] * cof[0][2];
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) {
    *err = "box is singular or non-finite";
    return NEP_ERR_ARG;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.Hinv[a][b] = cof[b][a] / det;
  *volume = std::fabs(det);
  double th[3];
  for (int a = 0; a < 3; ++a) {
    // face distance along axis a: |det| / |row b x row c| = 1 / |column a of Hinv|
    const double n = std::sqrt(g.Hinv[0][a] * g.Hinv[0][a] + g.Hinv[1][a] * g.Hinv[1][a] + g.Hinv[2][a] * g.Hinv[2][a]);
    th[a] = 1.0 / n;
    g.nc[a] = std::max(1, (int)std::floor(th[a] / rl));
  }
  // keep the grid no larger than about 4 cells per atom (coarser cells stay valid)
  const long long limit = std::max<long long>(64, 4LL * N);
  while ((long long)g.nc[0] * g.nc[1] * g.nc[2] > limit) {
    int a = 0;
    for (int b = 1; b < 3; ++b)
      if (g.nc[b] > g.nc[a]) a = b;
    g.nc[a] = std::max(1, g.nc[a] / 2);
  }
  int rmax = 0;
  for (int a = 0; a < 3; ++a) {
    g.R[a] = (int)std::ceil(rl * g.nc[a] / th[a] - 1e-12);
    if (g.R[a] < 1) g.R[a] = 1;
    rmax = std::max(rmax, g.R[a]);
    g.reach[a] = (float)((rl + kReachMargin) * g.nc[a] / th[a]);
  }
  if (rmax > kMaxImage) {
    *err = "cell thinner than a third of r_c^R + skin; replicate the cell before calling";
    return NEP_ERR_UNSUPPORTED;
  }
  g.ncell = g.nc[0] * g.nc[1] * g.nc[2];
  g.obits = rmax <= 1 ? 2 : 3;
  int jb = 1;
  while ((1LL << jb) < (long long)std::max(N, 2)) ++jb;
  if (jb + 3 * g.obits > 32) {
    *err = "too many atoms for the packed neighbour entries";
    return NEP_ERR_UNSUPPORTED;
  }
  g.jbits = jb;
  g.jmask = (jb >= 32) ? 0xffffffffu : ((1u << jb) - 1u);
  g.ncode = 1 << (3 * g.obits);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.Hc[a][b] = g.H[a][b] / g.nc[a];
  if (!dtab) return NEP_OK;
  for (int c = 0; c < g.ncode; ++c) dtab[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int ox = -g.R[0]; ox <= g.R[0]; ++ox)
    for (int oy = -g.R[1]; oy <= g.R[1]; ++oy)
      for (int oz = -g.R[2]; oz <= g.R[2]; ++oz) {
        const unsigned code = (unsigned)(ox + g.R[0]) | ((unsigned)(oy + g.R[1]) << g.obits) |
                              ((unsigned)(oz + g.R[2]) << (2 * g.obits));
        double D[3];
        for (int b = 0; b < 3; ++b) D[b] = ox * g.Hc[0][b] + oy * g.Hc[1][b] + oz * g.Hc[2][b];
        dtab[code] = make_float4((float)D[0], (float)D[1], (float)D[2], 0.f);
      }
  return NEP_OK;
}

// Validates the model parameters and finds the compiled kernel shape.
int check_params(const nep_params *p, const ShapeOps **ops_out, const char **err) {
  *ops_out = nullptr;
  if (!p) { *err = "params is null"; return NEP_ERR_ARG; }
  if (p->version != 3) { *err = "version must be 3"; return NEP_ERR_ARG; }
  if (p->n_types < 1 || p->n_types > NEP_MAX_TYPES) { *err = "n_types out of range"; return NEP_ERR_ARG; }
  if (!(p->rc_radial > 0) || !(p->rc_angular > 0) || p->rc_angular > p->rc_radial || !std::isfinite(p->rc_radial)) {
    *err = "need 0 < rc_angular <= rc_radial";
    return NEP_ERR_ARG;
  }
  if (p->n_max_radial < 0 || p->n_max_angular < 0 || p->basis_radial < 0 || p->basis_angular < 0 ||
      p->n_neuron < 1) {
    *err = "negative size";
    return NEP_ERR_ARG;
  }
  if (p->l_max_3b < 1 || p->l_max_3b > 4 || !(p->l_max_4b == 0 || p->l_max_4b == 2) ||
      !(p->l_max_5b == 0 || p->l_max_5b == 1)) {
    *err = "need l_max_3b in 1..4, l_max_4b in {0,2}, l_max_5b in {0,1}";
    return NEP_ERR_ARG;
  }
  if (!p->c_radial || !p->c_angular || !p->w0 || !p->b0 || !p->w1) {
    *err = "null weight pointer";
    return NEP_ERR_ARG;
  }
  for (int i = 0; i < shape_count(); ++i) {
    const ShapeOps *o = shape_at(i);
    if (o->nR == p->n_max_radial && o->KR == p->basis_radial && o->nA == p->n_max_angular &&
        o->KA == p->basis_angular && o->H == p->n_neuron && o->L3 == p->l_max_3b && o->L4 == p->l_max_4b &&
        o->L5 == p->l_max_5b)
      *ops_out = o;
  }
  if (!*ops_out) {
    // no compiled instantiation: the kernels that take the shape at run time
    if (p->n_max_radial > kGenMaxN || p->n_max_angular > kGenMaxN || p->basis_radial > kGenMaxN ||
        p->basis_angular > kGenMaxN || p->n_neuron > kGenMaxNeu) {
      *err = "shape beyond the limits of the run-time-shape kernels (n_max, N_bas <= 19, N_neu <= 256)";
      return NEP_ERR_UNSUPPORTED;
    }
    *ops_out = shape_generic();
  }
  return NEP_OK;
}

// Descriptor length N_des (Sec. II C) of a validated parameter set.
int n_des_of(const nep_params *p) {
  const int nb = p->l_max_3b + (p->l_max_4b >= 2 ? 1 : 0) + (p->l_max_5b >= 1 ? 1 : 0);
  return (p->n_max_radial + 1) + (p->n_max_angular + 1) * nb;
}

// Run-time shape fields of the kernel arguments (read only by the run-time-shape kernels).
void set_shape_args(AtomArgs &a, const nep_params &p, const float *ann) {
  a.gR = p.n_max_radial;
  a.gKR = p.basis_radial;
  a.gA = p.n_max_angular;
  a.gKA = p.basis_angular;
  a.gH = p.n_neuron;
  a.gL3 = p.l_max_3b;
  a.gL4 = p.l_max_4b;
  a.gL5 = p.l_max_5b;
  a.gD = n_des_of(&p);
  a.ann = ann;
}

}  // namespace nep

namespace {

const double kPi = 3.14159265358979323846;
// 1 u * A^2 / fs^2 in eV from the CODATA 2018 atomic mass unit and elementary charge.
const double kKappa = 1.66053906660e-27 * 1e-20 / 1e-30 / 1.602176634e-19;

enum Slot { SLOT_DRIFT = 0, SLOT_REBUILD, SLOT_ATOM, SLOT_GATHER, SLOT_FINAL, N_SLOTS };
const char *kSlotNames[N_SLOTS] = {"md_drift", "neighbor_rebuild", "nep_atom", "nep_gather", "finalize"};

thread_local std::string g_create_error;  // per calling thread (serving workers create handles)

// Device buffers of the calling thread are stream-ordered (cudaMallocAsync / cudaFreeAsync
// on this stream) when it is set: the serving workers use this so that growing or releasing
// a workspace never synchronises the device.
thread_local cudaStream_t t_alloc_stream = nullptr;
thread_local bool t_alloc_async = false;

// Wait for a stream. Threads in the stream-ordered mode (the serving workers, many per CPU
// core) poll with short sleeps instead of spinning in cudaStreamSynchronize.
cudaError_t wait_stream(cudaStream_t s) {
  if (!t_alloc_async) return cudaStreamSynchronize(s);
  for (;;) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e != cudaErrorNotReady) return e;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

template <class Tp>
struct DevBuf {
  Tp *p = nullptr;
  size_t n = 0;
  bool async = false;
  cudaStream_t st = nullptr;
  cudaError_t ensure(size_t want) {
    if (want <= n && p) return cudaSuccess;
    release();
    if (want == 0) want = 1;
    async = t_alloc_async;
    st = t_alloc_stream;
    cudaError_t e = async ? cudaMallocAsync(reinterpret_cast<void **>(&p), want * sizeof(Tp), st)
                          : cudaMalloc(reinterpret_cast<void **>(&p), want * sizeof(Tp));
    if (e == cudaSuccess) n = want;
    else p = nullptr;
    return e;
  }
  void release() {
    if (p) {
      if (async) cudaFreeAsync(p, st);
      else cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return p ? n * sizeof(Tp) : 0; }
};

}  // namespace

namespace nep {
void set_create_error(const char *msg) { g_create_error = msg ? msg : ""; }
}  // namespace nep

// Identity of a captured batch graph: every array it touches and the list capacities.
struct BatchKey {
  const void *p[16];
  long long gen;
  int N, cap_r, cap_a, precision, blocks, pad;
};

// Identity of a captured engine iteration: every array it touches and the list capacities.
struct EngineKey {
  const void *p[25];
  long long gen;
  int N, cap_r, cap_a, precision;
};

// Launch shapes of the batched kernels, set by the caller or the autotuner (0 = default).
struct Tuning {
  int members = 0;       // population members per launch (grid.y)
  int atom_block = 0;    // atoms per CTA of the batched atom kernel (64, 128)
  int gather_block = 0;  // atoms per CTA of the batched gather kernel (64, 128, 256)
  int last_members = 0;  // members per launch of the last population evaluation
  int n_tried = 0;       // candidates timed by the last autotune
  float best_ms = 0.f, default_ms = 0.f;  // per-evaluation times of the choice and of the defaults
  int atom_form = 0;     // FP32 per-atom kernel of nep_compute / md_run: 0 default, 1, 3 (AtomArgs.atom_occ)
};


struct nep_handle {
  // model
  int T = 0, nR = 0, nA = 0, KR = 0, KA = 0, L3 = 0, L4 = 0, L5 = 0, H = 0, n_des = 0;
  double rcR = 0, rcA = 0, skin = 1.0;
  std::vector<float> w0, b0, w1, cR, cA;
  float b1 = 0;
  std::vector<double> mass;
  ModelF mf;
  const ShapeOps *ops = nullptr;
  int device = 0;
  std::string err;
  // device model copies
  DevBuf<float> d_cR, d_cA;
  DevBuf<double> d_inv_mk, d_mk_half;
  // workspace
  int N = 0;
  int cap_r = 0, cap_a = 0;
  Grid grid;
  double volume = 0;
  DevBuf<double> x, v, F, x_ref, origin, partial_atom, partial_gather, thermo_stage;
  DevBuf<double> ck_x, ck_v, ck_F;  // md_run checkpoint (start of the current chunk)
  DevBuf<int> ck_types, ck_perm;
  DevBuf<double> x2, v2, F2;        // reorder scratch
  DevBuf<int> types2, perm2, cell2, perm;
  DevBuf<int> types, cell_of, cell_count, cell_cursor, cell_start, cell_atoms, nn_r, nn_a, rev_a, thermo_ctl;
  DevBuf<unsigned> nl_r, nl_a, stage_e;
  DevBuf<unsigned char> stage_g;
  DevBuf<float4> pos4, posA, dtab, p_ang;
  DevBuf<float> e_rad;
  DevBuf<BuildStatus> status;
  BuildStatus *h_status = nullptr;  // pinned mirror
  // md
  bool md_ready = false;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t fire_graph = nullptr;  // one FIRE step (its time step lives on the device)
  DevBuf<FireState> fire, ck_fire;
  DevBuf<ThermoState> thermo_state, ck_thermo;  // BDP thermostat (md_run_ex)
  // batched serving engine: one structure per job, all advanced by one iteration
  std::vector<EngineSlot> e_slots_h;            // host mirror (after the last iteration)
  std::vector<double> e_energy_h, e_virial_h;   // per job, after the last iteration
  DevBuf<EngineSlot> e_slots, e_slots_ck;
  DevBuf<int> e_sflag;  // per-job build requests of the drift kernel (partial builds)
  DevBuf<double> e_energy, e_virial, e_u, e_w, e_xck, e_vck;
  DevBuf<int4> e_table;
  cudaGraphExec_t e_graph = nullptr;            // one captured iteration of the current layout
  EngineKey e_key{}, e_last{};
  bool nvt = false;                             // the MD step graph rescales velocities
  bool graph_nvt = false;
  double graph_dt = 0;
  bool graph_prof = false;
  const double *graph_thermo = nullptr;
  cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
  int rebuild_kernels = 0;  // kernels in the conditional rebuild body of the step graph
  bool graph_cond = true;   // rebuild inside a conditional node (else early-exit kernel nodes)
  int precision = 0;        // network arithmetic: 0 FP32 SIMT, 1 BF16 tensor cores
  int graph_prec = 0;
  DevBuf<uint4> d_tc;       // BF16 W0 operand tiles for the tensor-core network
  DevBuf<float> d_ann;      // FP32 network [w0 | b0 | w1 | b1] (run-time-shape kernels)
  bool generic = false;     // no compiled instantiation of this shape
  bool graph_cond_used = true;
  // batches of structures: layout of the last batch (reused while unchanged)
  int nb_struct = 0;
  std::vector<int> b_offsets;
  std::vector<double> b_boxes;
  std::vector<Grid> b_grids;
  DevBuf<Grid> d_grids;
  DevBuf<int> d_sid, d_offsets;
  DevBuf<double> b_e, b_w;  // caller-order per-atom energies and virials when the caller keeps none
  long long b_gen = 0;      // layout generation (bumped when the grids change)
  cudaGraphExec_t b_graph = nullptr;
  int b_graph_kernels = 0;
  BatchKey b_key{}, b_last{};
  // population evaluation: per-member kernel arrays and the sums of Eq. loss
  DevBuf<float> pop_cr, pop_ca, pop_ann;
  DevBuf<uint4> pop_tc;
  DevBuf<double> pop_reg, pop_es, pop_ws;
  Tuning tune;
  // profiling
  bool prof = false;
  cudaEvent_t ev[N_SLOTS][2] = {};
  bool slot_ran[N_SLOTS] = {};
  nep_stats stats_cache{};
  int graph_kernels = 0;
  // every per-structure device buffer (not the model copies, the status word or the tiles)
  template <class Fn>
  void for_workspace(Fn &&f) {
    f(x); f(v); f(F); f(x_ref); f(origin); f(partial_atom); f(partial_gather); f(thermo_stage);
    f(ck_x); f(ck_v); f(ck_F); f(ck_types); f(ck_perm); f(x2); f(v2); f(F2); f(types2); f(perm2); f(cell2);
    f(perm); f(types); f(cell_of); f(cell_count); f(cell_cursor); f(cell_start); f(cell_atoms); f(nn_r);
    f(nn_a); f(rev_a); f(thermo_ctl); f(nl_r); f(nl_a); f(pos4); f(posA); f(dtab); f(p_ang); f(e_rad); f(d_grids);
    f(d_sid); f(d_offsets); f(b_e); f(b_w); f(pop_cr); f(pop_ca); f(pop_ann); f(pop_tc); f(pop_reg); f(pop_es);
    f(pop_ws); f(fire); f(ck_fire); f(thermo_state); f(ck_thermo); f(stage_e); f(stage_g); f(e_slots);
    f(e_slots_ck); f(e_energy); f(e_virial); f(e_u); f(e_w); f(e_xck); f(e_vck); f(e_table);
  }
  // the kernels compare r^2 with the FP32 square of the FP32 cutoff
  float rcR2f() const { return (float)rcR * (float)rcR; }
  float rcA2f() const { return (float)rcA * (float)rcA; }
};

namespace {

int fail(nep_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(nep_handle *h, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, NEP_ERR_OOM, std::string(where) + ": out of device memory");
  }
  return fail(h, NEP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

void ev_record(nep_handle *h, int slot, int which, cudaStream_t s, bool capturing) {
  if (!h->prof) return;
  if (capturing) cudaEventRecordWithFlags(h->ev[slot][which], s, cudaEventRecordExternal);
  else cudaEventRecord(h->ev[slot][which], s);
  if (which == 1) h->slot_ran[slot] = true;
}

int setup_grid(nep_handle *h, int N, const double *box, std::vector<float4> &dtab) {
  dtab.assign(1 << (3 * 3), make_float4(0.f, 0.f, 0.f, 0.f));
  const char *err = nullptr;
  const int rc = nep::build_grid(box, h->rcR + h->skin, N, h->grid, dtab.data(), &h->volume, &err);
  if (rc) return fail(h, rc, err);
  dtab.resize(h->grid.ncode);
  return NEP_OK;
}

int ensure_atoms(nep_handle *h, int N, cudaStream_t s) {
  const size_t n = (size_t)std::max(N, 1);
  CK(h->x.ensure(3 * n), "alloc");
  CK(h->v.ensure(3 * n), "alloc");
  CK(h->F.ensure(3 * n), "alloc");
  CK(h->x_ref.ensure(3 * n), "alloc");
  CK(h->origin.ensure(3 * n), "alloc");
  CK(h->types.ensure(n), "alloc");
  CK(h->cell_of.ensure(n), "alloc");
  CK(h->cell_atoms.ensure(n), "alloc");
  CK(h->pos4.ensure(n), "alloc");
  CK(h->posA.ensure(n), "alloc");
  CK(h->x2.ensure(3 * n), "alloc");
  CK(h->v2.ensure(3 * n), "alloc");
  CK(h->F2.ensure(3 * n), "alloc");
  CK(h->types2.ensure(n), "alloc");
  CK(h->perm2.ensure(n), "alloc");
  CK(h->cell2.ensure(n), "alloc");
  CK(h->perm.ensure(n), "alloc");
  CK(h->nn_r.ensure(n * h->T), "alloc");
  CK(h->nn_a.ensure(n), "alloc");
  CK(h->e_rad.ensure(n * h->T * (size_t)(((h->KR + 2) + 3) / 4 * 4)), "alloc");
  CK(h->partial_atom.ensure(h->ops->atom_blocks(N) + 1), "alloc");
  CK(h->partial_gather.ensure((size_t)(h->ops->gather_blocks(N) + 1) * kReduceSlots), "alloc");
  if (!h->status.p) {  // a new status word starts cleared (device memory comes uninitialised)
    CK(h->status.ensure(1), "alloc");
    CK(cudaMemsetAsync(h->status.p, 0, sizeof(BuildStatus), s), "clear status");
    std::memset(h->h_status, 0, sizeof(BuildStatus));
  }
  CK(h->thermo_ctl.ensure(4), "alloc");
  return NEP_OK;
}

int ensure_lists(nep_handle *h, int N, int cap_r, int cap_a) {
  const size_t n = (size_t)std::max(N, 1);
  CK(h->nl_r.ensure(n * cap_r), "alloc lists");
  CK(h->nl_a.ensure(n * cap_a), "alloc lists");
  CK(h->rev_a.ensure(n * cap_a), "alloc lists");
  CK(h->p_ang.ensure(n * cap_a), "alloc lists");
  CK(h->stage_e.ensure(n * cap_r), "alloc lists");
  CK(h->stage_g.ensure(n * cap_r), "alloc lists");
  h->cap_r = cap_r;
  h->cap_a = cap_a;
  return NEP_OK;
}

int read_status(nep_handle *h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost, s), "status");
  CK(wait_stream(s), "sync");
  return NEP_OK;
}

void reset_status_counts(nep_handle *h) {
  h->h_status->overflow = 0;
  h->h_status->max_r = 0;
  h->h_status->max_a = 0;
  h->h_status->rev_missing = 0;
  h->h_status->sum_r = 0;
  h->h_status->sum_a = 0;
  h->h_status->bad_input = 0;
  h->h_status->in_r = 0;
  h->h_status->in_a = 0;
  h->h_status->tc_timeout = 0;
}

AtomState atom_state(nep_handle *h) {
  AtomState a;
  a.x = h->x.p; a.v = h->v.p; a.F = h->F.p; a.x_ref = h->x_ref.p; a.origin = h->origin.p;
  a.types = h->types.p; a.perm = h->perm.p; a.cell_of = h->cell_of.p; a.pos4 = h->pos4.p; a.posA = h->posA.p;
  a.x2 = h->x2.p; a.v2 = h->v2.p; a.F2 = h->F2.p; a.types2 = h->types2.p; a.perm2 = h->perm2.p;
  a.cell2 = h->cell2.p;
  return a;
}

ListBufs list_bufs(nep_handle *h) {
  ListBufs L;
  L.cell_count = h->cell_count.p; L.cell_cursor = h->cell_cursor.p; L.cell_start = h->cell_start.p;
  L.cell_atoms = h->cell_atoms.p; L.nl_r = h->nl_r.p; L.nn_r = h->nn_r.p; L.nl_a = h->nl_a.p; L.nn_a = h->nn_a.p;
  L.rev_a = h->rev_a.p; L.cap_r = h->cap_r; L.cap_a = h->cap_a;
  L.stage_e = h->stage_e.p; L.stage_g = h->stage_g.p;
  return L;
}

// List capacity for a largest observed length m: room for the structure to densify
// (random-weight models do) before a regrow is needed.
int round_cap(int m) { return std::min(kListBuf, (2 * m + 16 + 3) / 4 * 4); }

// Bin, size and build the neighbour lists for the positions in h->x (forced rebuild).
int rebuild_lists(nep_handle *h, int N, cudaStream_t s, const Batch &B = Batch{nullptr, nullptr, 0}) {
  Grid &g = h->grid;
  CK(h->cell_count.ensure(g.ncell + 1), "alloc cells");
  CK(h->cell_cursor.ensure(g.ncell + 1), "alloc cells");
  CK(h->cell_start.ensure(g.ncell + 1), "alloc cells");
  const float rlR = (float)(h->rcR + h->skin), rlA = (float)(h->rcA + h->skin);
  for (int attempt = 0; attempt < 3; ++attempt) {
    const bool count_only = (h->cap_r == 0 || h->cap_a == 0);
    CK(cudaMemcpyAsync(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost, s), "status");
    CK(wait_stream(s), "sync");
    reset_status_counts(h);
    h->h_status->rebuild = 1;
    h->h_status->full = 1;
    CK(cudaMemcpyAsync(h->status.p, h->h_status, sizeof(BuildStatus), cudaMemcpyHostToDevice, s), "status");
    CK(launch_rebuild(N, h->T, g, B, h->dtab.p, rlR * rlR, rlA * rlA, h->rcR2f(), h->rcA2f(), atom_state(h),
                      list_bufs(h), count_only ? 1 : 0, h->status.p, s),
       "launch rebuild");
    CK(cudaGetLastError(), "launch rebuild");
    int rc = read_status(h, s);
    if (rc) return rc;
    const BuildStatus &st = *h->h_status;
    if (st.bad_input & 1) return fail(h, NEP_ERR_ARG, "atom type out of range");
    if (st.bad_input & 2) return fail(h, NEP_ERR_NONFINITE, "non-finite position");
    if (st.max_r > kListBuf || st.max_a > kListBuf)
      return fail(h, NEP_ERR_NEIGHBOR_OVERFLOW, "more than " + std::to_string(kListBuf) +
                                                    " neighbours within r_c + skin for one atom");
    if (count_only || st.overflow) {
      rc = ensure_lists(h, N, round_cap(std::max(1, st.max_r)), round_cap(std::max(1, st.max_a)));
      if (rc) return rc;
      continue;
    }
    if (st.rev_missing) return fail(h, NEP_ERR_CUDA, "angular neighbour list is not symmetric");
    h->stats_cache.max_radial = st.max_r;
    h->stats_cache.max_angular = st.max_a;
    h->stats_cache.mean_radial = N ? (double)st.sum_r / N : 0.0;
    h->stats_cache.mean_angular = N ? (double)st.sum_a / N : 0.0;
    h->stats_cache.mean_radial_in_rc = N ? (double)st.in_r / N : 0.0;
    h->stats_cache.mean_angular_in_rc = N ? (double)st.in_a / N : 0.0;
    return NEP_OK;
  }
  return fail(h, NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists could not be sized");
}

// The FP32 per-atom kernel form in use: the caller's choice, else the low-register form (3)
// where the shape has it (measured faster: 8.86 against 9.43 ms per step on 8,000,000 Si
// atoms), else 1.
int atom_form_of(const nep_handle *h) {
  const int f = h->tune.atom_form ? h->tune.atom_form : 3;
  return (f == 3 && h->ops && h->ops->lowreg) ? 3 : 1;
}

AtomArgs make_args(nep_handle *h, int N) {
  AtomArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = N;
  a.T = h->T;
  a.jbits = h->grid.jbits;
  a.jmask = h->grid.jmask;
  a.ncode = h->grid.ncode;
  a.rcR = (float)h->rcR;
  a.rcA = (float)h->rcA;
  a.pos4 = h->pos4.p;
  a.dtab = h->dtab.p;
  a.nl_r = h->nl_r.p;
  a.nn_r = h->nn_r.p;
  a.nl_a = h->nl_a.p;
  a.nn_a = h->nn_a.p;
  a.rev_a = h->rev_a.p;
  a.cap_r = h->cap_r;
  a.cap_a = h->cap_a;
  a.c_r = h->d_cR.p;
  a.c_a = h->d_cA.p;
  a.e_rad = h->e_rad.p;
  a.est = ((h->KR + 2) + 3) / 4 * 4;
  a.p_ang = h->p_ang.p;
  a.partial_atom = h->partial_atom.p;
  a.partial_gather = h->partial_gather.p;
  a.inv_mass_kappa = h->d_inv_mk.p;
  a.mass_kappa_half = h->d_mk_half.p;
  a.vel = h->v.p;
  a.perm = h->perm.p;
  a.precision = h->precision;
  a.tc_b1 = h->d_tc.p;
  a.tc_b2 = h->d_tc.p ? h->d_tc.p + (size_t)h->ops->np1 * h->ops->kp1 * 2 / 16 : nullptr;
  a.tc_err = h->status.p ? &h->status.p->tc_timeout : nullptr;
  a.gR = h->nR; a.gKR = h->KR; a.gA = h->nA; a.gKA = h->KA; a.gH = h->H;
  a.gL3 = h->L3; a.gL4 = h->L4; a.gL5 = h->L5; a.gD = h->n_des;
  a.ann = h->d_ann.p;
  a.atom_occ = atom_form_of(h);
  return a;
}

// Identity of the per-atom kernel a captured MD step uses (network form and FP32 kernel form).
int kernel_form(const nep_handle *h) {
  return h->precision * 16 + atom_form_of(h);
}

// Load positions (device, [N][3]) and types, set up the grid and build the lists.
int load_structure(nep_handle *h, int N, const double *pos, const int *types, const double *box, cudaStream_t s) {
  int rc = ensure_atoms(h, N, s);
  if (rc) return rc;
  std::vector<float4> dtab;
  rc = setup_grid(h, N, box, dtab);
  if (rc) return rc;
  CK(h->dtab.ensure(dtab.size()), "alloc");
  CK(cudaMemcpyAsync(h->dtab.p, dtab.data(), dtab.size() * sizeof(float4), cudaMemcpyHostToDevice, s), "copy");
  CK(cudaMemcpyAsync(h->x.p, pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy pos");
  CK(cudaMemcpyAsync(h->types.p, types, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "copy types");
  launch_iota(N, h->perm.p, s);
  h->N = N;
  h->stats_cache.n_atoms = N;
  for (int a = 0; a < 3; ++a) h->stats_cache.cells[a] = h->grid.nc[a];
  return rebuild_lists(h, N, s);
}

// Outputs for the caller (nep_compute) are scattered to the caller's atom order; the MD
// forces (force == h->F) stay in the internal order.
int run_forces(nep_handle *h, int N, double *energy, double *force, double *virial, int md_kick, double half_dt,
               cudaStream_t s, bool capturing, const FireState *fire = nullptr) {
  AtomArgs a = make_args(h, N);
  a.fire = fire;
  if (force == h->F.p) a.perm = nullptr;
  a.energy = energy;
  a.force = force;
  a.virial = virial;
  a.md_kick = md_kick;
  a.half_dt = half_dt;
  ev_record(h, SLOT_ATOM, 0, s, capturing);
  cudaError_t e = h->ops->atom(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, 0, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "nep_atom kernel");
  ev_record(h, SLOT_ATOM, 1, s, capturing);
  ev_record(h, SLOT_GATHER, 0, s, capturing);
  e = h->ops->gather(a, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "nep_gather kernel");
  ev_record(h, SLOT_GATHER, 1, s, capturing);
  return NEP_OK;
}

bool valid_handle(const nep_handle *h) { return h && h->ops; }

// Grids of all structures of a batch: each structure has its own cell grid and image
// range; the cells are numbered structure by structure, the shift tables share one code
// width (the largest), and list entries one atom-index width (for the whole batch).
int setup_batch(nep_handle *h, int n_struct, const int *offsets, const double *boxes, int N, cudaStream_t s) {
  int rc = ensure_atoms(h, N, s);
  if (rc) return rc;
  const bool same = n_struct == h->nb_struct && (int)h->b_offsets.size() == n_struct + 1 &&
                    std::equal(offsets, offsets + n_struct + 1, h->b_offsets.begin()) &&
                    std::equal(boxes, boxes + 9 * (size_t)n_struct, h->b_boxes.begin());
  if (!same) {
    h->nb_struct = 0;
    std::vector<Grid> &G = h->b_grids;
    G.assign(n_struct, Grid{});
    int obits = 2;
    for (int k = 0; k < n_struct; ++k) {
      const char *err = nullptr;
      double vol = 0;
      rc = nep::build_grid(boxes + 9 * (size_t)k, h->rcR + h->skin, std::max(offsets[k + 1] - offsets[k], 1), G[k],
                           nullptr, &vol, &err);
      if (rc) return fail(h, rc, "structure " + std::to_string(k) + ": " + err);
      obits = std::max(obits, G[k].obits);
    }
    int jb = 1;
    while ((1LL << jb) < (long long)std::max(N, 2)) ++jb;
    if (jb + 3 * obits > 32) return fail(h, NEP_ERR_UNSUPPORTED, "too many atoms for the packed neighbour entries");
    if (n_struct > (1 << 23)) return fail(h, NEP_ERR_UNSUPPORTED, "more than 2^23 structures");
    const int ncode = 1 << (3 * obits);
    long long ncell = 0;
    for (int k = 0; k < n_struct; ++k) {
      Grid &g = G[k];
      g.obits = obits;
      g.ncode = ncode;
      g.jbits = jb;
      g.jmask = (jb >= 32) ? 0xffffffffu : ((1u << jb) - 1u);
      g.cell_off = (int)ncell;
      g.dtab_off = k * ncode;
      ncell += g.ncell;
      if (ncell > (1LL << 30)) return fail(h, NEP_ERR_UNSUPPORTED, "too many cells in the batch");
    }
    Grid gg = G[0];  // batch-wide fields: cell count, entry packing
    gg.ncell = (int)ncell;
    gg.cell_off = 0;
    gg.dtab_off = 0;
    h->grid = gg;
    CK(h->d_grids.ensure(n_struct), "alloc batch");
    CK(h->d_offsets.ensure(n_struct + 1), "alloc batch");
    CK(h->dtab.ensure((size_t)n_struct * ncode), "alloc batch");
    // the copies read the handle's own host arrays, which change only at the next layout
    // (every caller synchronises the stream before that)
    h->b_offsets.assign(offsets, offsets + n_struct + 1);
    h->b_boxes.assign(boxes, boxes + 9 * (size_t)n_struct);
    CK(cudaMemcpyAsync(h->d_grids.p, G.data(), sizeof(Grid) * n_struct, cudaMemcpyHostToDevice, s), "copy grids");
    CK(cudaMemcpyAsync(h->d_offsets.p, h->b_offsets.data(), sizeof(int) * (n_struct + 1), cudaMemcpyHostToDevice, s),
       "copy offsets");
    launch_shift_tables(n_struct, h->d_grids.p, ncode, obits, h->dtab.p, s);
    h->b_gen += 1;
    h->nb_struct = n_struct;
  }
  CK(h->d_sid.ensure(std::max(N, 1)), "alloc batch");
  launch_struct_ids(n_struct, h->d_offsets.p, h->d_sid.p, s);
  CK(cudaGetLastError(), "batch setup");
  return NEP_OK;
}

// The largest structure of the batch layout (atoms).
int max_struct_atoms(const nep_handle *h) {
  int mx = 0;
  for (size_t k = 1; k < h->b_offsets.size(); ++k) mx = std::max(mx, h->b_offsets[k] - h->b_offsets[k - 1]);
  return mx;
}

Batch batch_of(nep_handle *h) {
  Batch B;
  B.grids = h->d_grids.p;
  B.sid = h->d_sid.p;
  B.n = h->nb_struct;
  return B;
}

// Kernel nodes of a graph (top level).
int count_kernel_nodes(cudaGraph_t graph) {
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
  int nk = 0;
  for (size_t k = 0; k < nn; ++k) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
  }
  return nk;
}

// Arrays of one batched evaluation.
struct BatchOut {
  const double *pos = nullptr;
  const int *types = nullptr;
  double *e_atom = nullptr, *w_atom = nullptr, *force = nullptr, *e_struct = nullptr, *w_struct = nullptr;
};

int atom_block(const nep_handle *h) { return (h->precision >= 1 || h->tune.atom_block == 0) ? 128 : h->tune.atom_block; }
int gather_block(const nep_handle *h) { return h->tune.gather_block == 0 ? 128 : h->tune.gather_block; }

// Per-block partial sums of `members` batched evaluations.
int ensure_partials(nep_handle *h, int N, int members) {
  const size_t nb_a = (N + atom_block(h) - 1) / atom_block(h), nb_g = (N + gather_block(h) - 1) / gather_block(h);
  CK(h->partial_atom.ensure((size_t)members * nb_a + 1), "alloc");
  CK(h->partial_gather.ensure(((size_t)members * nb_g + 1) * kReduceSlots), "alloc");
  return NEP_OK;
}

// Queue atom kernel, gather kernel and structure sums of a batch whose lists are built.
int batch_kernels(nep_handle *h, int N, const BatchOut &o, cudaStream_t s, bool capturing) {
  int rc = ensure_partials(h, N, 1);
  if (rc) return rc;
  AtomArgs a = make_args(h, N);
  a.energy = o.e_atom;
  a.force = o.force;
  a.virial = o.w_atom;
  a.s_out = N;
  ev_record(h, SLOT_ATOM, 0, s, capturing);
  cudaError_t e =
      h->ops->atom_batch(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, 1, atom_block(h), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "nep_atom kernel (batch)");
  ev_record(h, SLOT_ATOM, 1, s, capturing);
  ev_record(h, SLOT_GATHER, 0, s, capturing);
  e = h->ops->gather_batch(a, 1, gather_block(h), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "nep_gather kernel (batch)");
  ev_record(h, SLOT_GATHER, 1, s, capturing);
  ev_record(h, SLOT_FINAL, 0, s, capturing);
  if (o.e_struct || o.w_struct)
    launch_struct_sums(h->nb_struct, 1, h->d_offsets.p, N, o.e_struct ? o.e_atom : nullptr,
                       o.w_struct ? o.w_atom : nullptr, o.e_struct, o.w_struct, max_struct_atoms(h), s);
  ev_record(h, SLOT_FINAL, 1, s, capturing);
  CK(cudaGetLastError(), "structure sums");
  return NEP_OK;
}

BatchKey batch_key(nep_handle *h, int N, const BatchOut &o) {
  BatchKey k;
  std::memset(&k, 0, sizeof(k));
  const void *p[] = {o.pos, o.types, o.e_atom, o.w_atom, o.force, o.e_struct, o.w_struct, h->nl_r.p, h->nl_a.p,
                     h->rev_a.p, h->p_ang.p, h->e_rad.p, h->x.p, h->dtab.p, h->d_grids.p, h->cell_start.p};
  static_assert(sizeof(p) / sizeof(p[0]) == sizeof(k.p) / sizeof(k.p[0]), "key size");
  for (size_t c = 0; c < sizeof(p) / sizeof(p[0]); ++c) k.p[c] = p[c];
  k.gen = h->b_gen;
  k.N = N;
  k.cap_r = h->cap_r;
  k.cap_a = h->cap_a;
  k.precision = kernel_form(h);
  k.blocks = atom_block(h) * 1024 + gather_block(h);
  return k;
}

// Capture copy-in, forced neighbour build, kernels, structure sums and the status read of a
// batch into one graph (replayed by the next identical call).
int capture_batch(nep_handle *h, int N, const BatchOut &o, cudaStream_t s) {
  if (h->b_graph) {
    cudaGraphExecDestroy(h->b_graph);
    h->b_graph = nullptr;
  }
  std::memset(&h->b_key, 0, sizeof(h->b_key));
  CK(wait_stream(s), "sync");
  cudaStream_t c = h->cap_stream;
  CK(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "capture");
  cudaMemcpyAsync(h->x.p, o.pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, c);
  cudaMemcpyAsync(h->types.p, o.types, sizeof(int) * N, cudaMemcpyDeviceToDevice, c);
  launch_iota(N, h->perm.p, c);
  launch_arm_rebuild(h->status.p, c);
  const float rlR = (float)(h->rcR + h->skin), rlA = (float)(h->rcA + h->skin);
  cudaError_t e = launch_rebuild(N, h->T, h->grid, batch_of(h), h->dtab.p, rlR * rlR, rlA * rlA, h->rcR2f(),
                                 h->rcA2f(), atom_state(h), list_bufs(h), 0, h->status.p, c);
  int rc = e == cudaSuccess ? batch_kernels(h, N, o, c, true) : cuda_fail(h, e, "batch rebuild");
  if (!rc) cudaMemcpyAsync(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost, c);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(c, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture (batch)");
  h->b_graph_kernels = count_kernel_nodes(graph);
  e = cudaGraphInstantiate(&h->b_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->b_graph = nullptr;
    return cuda_fail(h, e, "graph instantiate (batch)");
  }
  return NEP_OK;
}

int check_offsets(nep_handle *h, int n_struct, const int *offsets) {
  if (n_struct < 0 || !offsets) return fail(h, NEP_ERR_ARG, "n_struct < 0 or offsets is null");
  if (offsets[0] != 0) return fail(h, NEP_ERR_ARG, "offsets[0] must be 0");
  for (int k = 0; k < n_struct; ++k)
    if (offsets[k + 1] < offsets[k]) return fail(h, NEP_ERR_ARG, "offsets must be non-decreasing");
  return NEP_OK;
}

}  // namespace

namespace nep {
void set_thread_alloc_stream(cudaStream_t s) {
  t_alloc_stream = s;
  t_alloc_async = s != nullptr;
}

void release_workspace(nep_handle *h) {
  for (cudaGraphExec_t *g : {&h->graph, &h->fire_graph, &h->b_graph})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  h->for_workspace([](auto &b) { b.release(); });
  h->N = 0;
  h->cap_r = h->cap_a = 0;
  h->md_ready = false;
  h->nb_struct = 0;
  h->b_offsets.clear();
  h->b_boxes.clear();
  std::memset(&h->b_key, 0, sizeof(h->b_key));
  std::memset(&h->b_last, 0, sizeof(h->b_last));
}

cudaError_t stream_sync(cudaStream_t s) { return wait_stream(s); }

// ---------------------------------------------------------------- batched serving engine
int engine_jobs(const nep_handle *h) { return h->nb_struct; }
int engine_atoms(const nep_handle *h) { return h->N; }
const EngineSlot &engine_slot(const nep_handle *h, int k) { return h->e_slots_h[k]; }
double engine_energy(const nep_handle *h, int k) { return h->e_energy_h[k]; }
const double *engine_virial(const nep_handle *h, int k) { return h->e_virial_h.data() + 9 * (size_t)k; }

// New job layout: the kept jobs (indices into the current layout, in order) and then the
// added ones. The atoms of every job stay contiguous; new jobs start at phase 0 (their first
// iteration evaluates their forces).
int engine_relayout(nep_handle *h, const std::vector<int> &keep, const std::vector<EngineJob> &add, cudaStream_t s,
                    size_t target_bytes) {
  const int S_old = h->nb_struct;
  std::vector<int> off_new(1, 0);
  std::vector<double> boxes;
  std::vector<EngineSlot> slots;
  std::vector<int4> table;
  for (int k : keep) {
    if (k < 0 || k >= S_old) return fail(h, NEP_ERR_ARG, "engine: bad job index");
    const int n = h->b_offsets[k + 1] - h->b_offsets[k];
    table.push_back(make_int4(h->b_offsets[k], off_new.back(), n, off_new.back() - h->b_offsets[k]));
    off_new.push_back(off_new.back() + n);
    boxes.insert(boxes.end(), h->b_boxes.begin() + 9 * (size_t)k, h->b_boxes.begin() + 9 * (size_t)k + 9);
    slots.push_back(h->e_slots_h[k]);
  }
  const int first_new = (int)slots.size();
  for (const EngineJob &j : add) {
    off_new.push_back(off_new.back() + j.n);
    boxes.insert(boxes.end(), j.box, j.box + 9);
    EngineSlot sl{};
    sl.kind = j.kind;
    sl.phase = 0;
    sl.n_steps = j.kind == kJobSingle ? 0 : j.n_steps;
    sl.dt = j.dt;
    if (j.kind == kJobFire) {
      sl.fire.dt = j.dt;
      sl.fire.alpha = 0.1;
      sl.fire.dt_max = 10.0 * j.dt;
      sl.fire.fmax2 = j.fmax * j.fmax;
    }
    slots.push_back(sl);
  }
  const int S_new = (int)slots.size(), N_new = off_new.back();
  // move the kept jobs into the reorder scratch arrays, fill in the new ones, swap
  const size_t n = (size_t)std::max(N_new, 1);
  CK(h->x2.ensure(3 * n), "alloc");
  CK(h->v2.ensure(3 * n), "alloc");
  CK(h->F2.ensure(3 * n), "alloc");
  CK(h->types2.ensure(n), "alloc");
  CK(h->perm2.ensure(n), "alloc");
  AtomState dst = atom_state(h);
  dst.x = h->x2.p; dst.v = h->v2.p; dst.F = h->F2.p; dst.types = h->types2.p; dst.perm = h->perm2.p;
  if (!table.empty()) {
    CK(h->e_table.ensure(table.size()), "alloc");
    CK(cudaMemcpyAsync(h->e_table.p, table.data(), sizeof(int4) * table.size(), cudaMemcpyHostToDevice, s), "copy");
    launch_engine_relayout((int)table.size(), h->e_table.p, atom_state(h), dst, s);
  }
  if (!add.empty()) {
    // the new jobs are contiguous at the end of the layout: one copy per array
    const size_t o0 = (size_t)off_new[first_new], na = (size_t)N_new - o0;
    std::vector<double> px(3 * na), pv(3 * na, 0.0);
    std::vector<int> pt(na), pp(na);
    for (size_t a = 0; a < add.size(); ++a) {
      const EngineJob &j = add[a];
      const size_t o = (size_t)off_new[first_new + a] - o0;
      std::memcpy(px.data() + 3 * o, j.pos, sizeof(double) * 3 * j.n);
      if (j.vel) std::memcpy(pv.data() + 3 * o, j.vel, sizeof(double) * 3 * j.n);
      std::memcpy(pt.data() + o, j.types, sizeof(int) * j.n);
      for (int k = 0; k < j.n; ++k) pp[o + k] = (int)(o0 + o) + k;
    }
    CK(cudaMemcpyAsync(dst.x + 3 * o0, px.data(), sizeof(double) * 3 * na, cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemcpyAsync(dst.v + 3 * o0, pv.data(), sizeof(double) * 3 * na, cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemsetAsync(dst.F + 3 * o0, 0, sizeof(double) * 3 * na, s), "zero");
    CK(cudaMemcpyAsync(dst.types + o0, pt.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemcpyAsync(dst.perm + o0, pp.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s), "copy");
    CK(wait_stream(s), "sync");  // the host staging vectors are temporaries
  }
  std::swap(h->x, h->x2);
  std::swap(h->v, h->v2);
  std::swap(h->F, h->F2);
  std::swap(h->types, h->types2);
  std::swap(h->perm, h->perm2);
  // buffers sized for an earlier, larger batch are released (and the lists sized again) when
  // the workspace exceeds the new batch's budget; only the batch state above is kept
  if (target_bytes && workspace_bytes(h) > target_bytes) {
    h->for_workspace([&](auto &b) {
      const void *p = b.p;
      if (p != h->x.p && p != h->v.p && p != h->F.p && p != h->types.p && p != h->perm.p) b.release();
    });
    h->cap_r = h->cap_a = 0;
    h->nb_struct = 0;
    h->b_offsets.clear();
    h->b_boxes.clear();
  }
  h->e_slots_h = slots;
  h->e_energy_h.assign(S_new, 0.0);
  h->e_virial_h.assign(9 * (size_t)S_new, 0.0);
  h->md_ready = false;
  for (cudaGraphExec_t *g : {&h->graph, &h->fire_graph, &h->b_graph, &h->e_graph})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  std::memset(&h->e_key, 0, sizeof(h->e_key));
  std::memset(&h->e_last, 0, sizeof(h->e_last));
  h->N = N_new;
  if (S_new == 0) {
    h->nb_struct = 0;
    h->b_offsets.assign(1, 0);
    h->b_boxes.clear();
    return NEP_OK;
  }
  int rc = ensure_atoms(h, N_new, s);
  if (rc) return rc;
  CK(h->e_slots.ensure(S_new), "alloc");
  CK(h->e_slots_ck.ensure(S_new), "alloc");
  CK(h->e_sflag.ensure(S_new), "alloc");
  CK(cudaMemsetAsync(h->e_sflag.p, 0, sizeof(int) * S_new, s), "clear build requests");
  CK(h->e_energy.ensure(S_new), "alloc");
  CK(h->e_virial.ensure(9 * (size_t)S_new), "alloc");
  CK(h->e_u.ensure(n), "alloc");
  CK(h->e_w.ensure(9 * n), "alloc");
  CK(h->e_xck.ensure(3 * n), "alloc");
  CK(h->e_vck.ensure(3 * n), "alloc");
  CK(cudaMemcpyAsync(h->e_slots.p, slots.data(), sizeof(EngineSlot) * S_new, cudaMemcpyHostToDevice, s), "copy");
  rc = setup_batch(h, S_new, off_new.data(), boxes.data(), N_new, s);
  if (rc) return rc;
  // the first layout sizes the lists with a counting pass; later ones keep the capacity (an
  // iteration whose build overflows is undone and run again with grown lists)
  if (h->cap_r == 0 || h->cap_a == 0) return rebuild_lists(h, N_new, s, batch_of(h));
  CK(h->cell_count.ensure(h->grid.ncell + 1), "alloc cells");
  CK(h->cell_cursor.ensure(h->grid.ncell + 1), "alloc cells");
  CK(h->cell_start.ensure(h->grid.ncell + 1), "alloc cells");
  return ensure_lists(h, N_new, h->cap_r, h->cap_a);
}

EngineKey engine_key(nep_handle *h) {
  EngineKey k;
  std::memset(&k, 0, sizeof(k));
  const void *p[] = {h->x.p, h->v.p, h->F.p, h->x_ref.p, h->origin.p, h->types.p, h->perm.p, h->pos4.p, h->posA.p,
                     h->nl_r.p, h->nl_a.p, h->rev_a.p, h->p_ang.p, h->e_rad.p, h->e_u.p, h->e_w.p, h->e_slots.p,
                     h->e_energy.p, h->d_grids.p, h->d_sid.p, h->dtab.p, h->cell_start.p, h->stage_e.p,
                     h->partial_gather.p, h->e_sflag.p};
  static_assert(sizeof(p) / sizeof(p[0]) == sizeof(k.p) / sizeof(k.p[0]), "key size");
  for (size_t c = 0; c < sizeof(p) / sizeof(p[0]); ++c) k.p[c] = p[c];
  k.gen = h->b_gen;
  k.N = h->N;
  k.cap_r = h->cap_r;
  k.cap_a = h->cap_a;
  k.precision = kernel_form(h);
  return k;
}

int engine_queue_iteration(nep_handle *h, cudaStream_t s);

// Capture one engine iteration of the current layout into a graph.
int capture_engine(nep_handle *h, cudaStream_t s) {
  if (h->e_graph) {
    cudaGraphExecDestroy(h->e_graph);
    h->e_graph = nullptr;
  }
  CK(wait_stream(s), "sync");
  cudaStream_t c = h->cap_stream;
  CK(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "capture");
  int rc = engine_queue_iteration(h, c);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture (engine)");
  e = cudaGraphInstantiate(&h->e_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->e_graph = nullptr;
    return cuda_fail(h, e, "graph instantiate (engine)");
  }
  return NEP_OK;
}

// Queue one iteration of every job: drift (requesting a neighbour build when an atom moved
// more than skin/2 since the last one), the build (its kernels return at once unless one is
// pending), forces, kick, FIRE update, bookkeeping (the per-job sums follow once per chunk).
int engine_queue_iteration(nep_handle *h, cudaStream_t s) {
  const int N = h->N, S = h->nb_struct;
  const float rlR = (float)(h->rcR + h->skin), rlA = (float)(h->rcA + h->skin);
  launch_engine_drift(N, atom_state(h), h->d_sid.p, h->e_slots.p, h->d_inv_mk.p, 0.25 * h->skin * h->skin,
                      h->e_sflag.p, h->status.p, s);
  // a build requested by the drift re-lists only the flagged jobs; a forced one every job
  Batch B = batch_of(h);
  B.sflag = h->e_sflag.p;
  cudaError_t e = launch_rebuild(N, h->T, h->grid, B, h->dtab.p, rlR * rlR, rlA * rlA, h->rcR2f(), h->rcA2f(),
                                 atom_state(h), list_bufs(h), 0, h->status.p, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "engine rebuild");
  AtomArgs a = make_args(h, N);
  a.perm = nullptr;  // every output in the internal order
  a.energy = h->e_u.p;
  a.force = h->F.p;
  a.virial = h->e_w.p;
  a.s_out = N;
  a.slots = h->e_slots.p;
  e = h->ops->atom_batch(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, 1, atom_block(h), s);
  if (e == cudaSuccess) e = h->ops->gather_batch(a, 1, gather_block(h), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "engine kernels");
  launch_engine_fire(S, h->d_offsets.p, atom_state(h), h->e_slots.p, s);
  launch_engine_advance(S, h->e_slots.p, s);
  CK(cudaGetLastError(), "engine step");
  return NEP_OK;
}

// n_iter iterations of every job (the first with a forced neighbour build after a new
// layout), then the per-job state is read back. The iterations start from a checkpoint: a
// list overflow in any of them undoes them all, grows the lists and runs them again. An
// unchanged layout replays one captured iteration graph.
int engine_step(nep_handle *h, cudaStream_t s, int n_iter, bool force_rebuild) {
  nep::NvtxRange nvtx_range("engine_step");
  const int N = h->N, S = h->nb_struct;
  if (N == 0 || S == 0 || n_iter < 1) return NEP_OK;
  CK(h->ck_F.ensure(3 * (size_t)N), "alloc checkpoint");
  CK(h->ck_types.ensure((size_t)N), "alloc checkpoint");
  CK(h->ck_perm.ensure((size_t)N), "alloc checkpoint");
  CK(h->ck_x.ensure(3 * (size_t)N), "alloc checkpoint");
  int rc = ensure_partials(h, N, 1);
  if (rc) return rc;
  for (int attempt = 0;; ++attempt) {
    // a build re-sorts the atoms: the checkpoint holds every per-atom array (x_ref too)
    CK(cudaMemcpyAsync(h->e_xck.p, h->x.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->e_vck.p, h->v.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_F.p, h->F.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_x.p, h->x_ref.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_types.p, h->types.p, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_perm.p, h->perm.p, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->e_slots_ck.p, h->e_slots.p, sizeof(EngineSlot) * S, cudaMemcpyDeviceToDevice, s),
       "checkpoint");
    const bool forced = force_rebuild || attempt > 0;
    // the flags of this chunk start cleared; a forced build is requested before the first step
    if (forced) launch_arm_rebuild(h->status.p, s);
    else launch_clear_flags(h->status.p, s);
    const EngineKey key = engine_key(h);
    for (int it = 0; it < n_iter; ++it) {
      if (!h->prof && h->e_graph && std::memcmp(&key, &h->e_key, sizeof(key)) == 0) {
        CK(cudaGraphLaunch(h->e_graph, s), "engine graph launch");
        continue;
      }
      if (!h->prof && std::memcmp(&key, &h->e_last, sizeof(key)) == 0) {
        // the layout was stable for a whole chunk: capture one iteration for the next ones
        rc = capture_engine(h, s);
        if (rc) return rc;
        h->e_key = key;
        CK(cudaGraphLaunch(h->e_graph, s), "engine graph launch");
        continue;
      }
      rc = engine_queue_iteration(h, s);
      if (rc) return rc;
    }
    h->e_last = key;
    // the jobs' energies and virials, once per chunk: only a job that finished (frozen since,
    // its per-atom values unchanged) or the chunk's last state is ever read
    launch_struct_sums(S, 1, h->d_offsets.p, N, h->e_u.p, h->e_w.p, h->e_energy.p, h->e_virial.p,
                       max_struct_atoms(h), s);
    CK(cudaMemcpyAsync(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost, s), "status");
    CK(wait_stream(s), "sync");
    const BuildStatus st = *h->h_status;
    if (st.tc_timeout) return fail(h, NEP_ERR_TIMEOUT, "a tensor-core completion wait ran out");
    if (st.bad_input & 2) return fail(h, NEP_ERR_NONFINITE, "non-finite position");
    if (st.bad_input & 1) return fail(h, NEP_ERR_ARG, "atom type out of range");
    if (!st.overflow && !st.rev_missing) break;
    if (attempt >= 2 || st.max_r > kListBuf || st.max_a > kListBuf)
      return fail(h, NEP_ERR_NEIGHBOR_OVERFLOW, "more than " + std::to_string(kListBuf) +
                                                    " neighbours within r_c + skin for one atom");
    CK(cudaMemcpyAsync(h->x.p, h->e_xck.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->v.p, h->e_vck.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->F.p, h->ck_F.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->x_ref.p, h->ck_x.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->types.p, h->ck_types.p, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->perm.p, h->ck_perm.p, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemcpyAsync(h->e_slots.p, h->e_slots_ck.p, sizeof(EngineSlot) * S, cudaMemcpyDeviceToDevice, s),
       "restore");
    int rc2 = ensure_lists(h, N, round_cap(st.max_r), round_cap(st.max_a));
    if (rc2) return rc2;
  }
  std::vector<EngineSlot> sl(S);
  CK(cudaMemcpyAsync(sl.data(), h->e_slots.p, sizeof(EngineSlot) * S, cudaMemcpyDeviceToHost, s), "read back");
  CK(cudaMemcpyAsync(h->e_energy_h.data(), h->e_energy.p, sizeof(double) * S, cudaMemcpyDeviceToHost, s), "read back");
  CK(cudaMemcpyAsync(h->e_virial_h.data(), h->e_virial.p, sizeof(double) * 9 * S, cudaMemcpyDeviceToHost, s),
     "read back");
  CK(wait_stream(s), "sync");
  h->e_slots_h = sl;
  return NEP_OK;
}

long long engine_builds(const nep_handle *h) { return h->h_status ? h->h_status->n_rebuilds : 0; }

// Final arrays of job k in its own atom order: positions wrapped into its cell, forces,
// velocities (HOST buffers [n][3], any may be null).
int engine_fetch(nep_handle *h, int k, double *pos, double *force, double *vel, cudaStream_t s) {
  if (k < 0 || k >= h->nb_struct) return fail(h, NEP_ERR_ARG, "engine: bad job index");
  const int o = h->b_offsets[k], n = h->b_offsets[k + 1] - o;
  std::vector<double> x(3 * (size_t)n), f(3 * (size_t)n), v(3 * (size_t)n);
  std::vector<int> perm(n);
  CK(cudaMemcpyAsync(x.data(), h->x.p + 3 * (size_t)o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaMemcpyAsync(f.data(), h->F.p + 3 * (size_t)o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaMemcpyAsync(v.data(), h->v.p + 3 * (size_t)o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaMemcpyAsync(perm.data(), h->perm.p + o, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "read");
  CK(wait_stream(s), "sync");
  const Grid &g = h->b_grids[k];
  for (int i = 0; i < n; ++i) {
    const int t = perm[i] - o;
    if (t < 0 || t >= n) return fail(h, NEP_ERR_CUDA, "engine: inconsistent atom order");
    double sf[3];
    for (int b = 0; b < 3; ++b) {
      sf[b] = x[3 * i] * g.Hinv[0][b] + x[3 * i + 1] * g.Hinv[1][b] + x[3 * i + 2] * g.Hinv[2][b];
      sf[b] -= std::floor(sf[b]);
    }
    for (int b = 0; b < 3; ++b) {
      if (pos) pos[3 * t + b] = sf[0] * g.H[0][b] + sf[1] * g.H[1][b] + sf[2] * g.H[2][b];
      if (force) force[3 * t + b] = f[3 * i + b];
      if (vel) vel[3 * t + b] = v[3 * i + b];
    }
  }
  return NEP_OK;
}

size_t workspace_bytes(nep_handle *h) {
  size_t t = 0;
  h->for_workspace([&](auto &b) { t += b.bytes(); });
  return t;
}
}  // namespace nep

// ======================================================================== C ABI
extern "C" {

int nep_supported(int *shapes, int max) {
  const int n = shape_count();
  for (int i = 0; i < n && i < max && shapes; ++i) {
    const ShapeOps *o = shape_at(i);
    int *r = shapes + 8 * i;
    r[0] = o->nR; r[1] = o->KR; r[2] = o->nA; r[3] = o->KA; r[4] = o->H; r[5] = o->L3; r[6] = o->L4; r[7] = o->L5;
  }
  return n;
}

int nep_create(const nep_params *p, nep_handle **out) {
  if (!out) return fail(nullptr, NEP_ERR_ARG, "out is null");
  *out = nullptr;
  const ShapeOps *ops = nullptr;
  const char *perr = nullptr;
  const int prc = check_params(p, &ops, &perr);
  if (prc) return fail(nullptr, prc, perr);
  nep_handle *h = new nep_handle();
  h->ops = ops;
  h->T = p->n_types; h->nR = p->n_max_radial; h->nA = p->n_max_angular; h->KR = p->basis_radial;
  h->KA = p->basis_angular; h->L3 = p->l_max_3b; h->L4 = p->l_max_4b; h->L5 = p->l_max_5b; h->H = p->n_neuron;
  h->n_des = n_des_of(p);
  h->generic = ops == shape_generic();
  h->rcR = p->rc_radial;
  h->rcA = p->rc_angular;
  h->skin = p->skin > 0 ? p->skin : 1.0;
  const int T = h->T;
  auto copyf = [](const double *src, size_t n, std::vector<float> &dst) {
    dst.resize(n);
    for (size_t k = 0; k < n; ++k) dst[k] = (float)src[k];
  };
  copyf(p->c_radial, (size_t)T * T * (h->nR + 1) * (h->KR + 1), h->cR);
  copyf(p->c_angular, (size_t)T * T * (h->nA + 1) * (h->KA + 1), h->cA);
  copyf(p->w0, (size_t)h->H * h->n_des, h->w0);
  copyf(p->b0, h->H, h->b0);
  copyf(p->w1, h->H, h->w1);
  h->b1 = (float)p->b1;
  for (float v : h->w0) if (!std::isfinite(v)) { delete h; return fail(nullptr, NEP_ERR_ARG, "non-finite weight"); }
  if (p->mass) {
    h->mass.assign(p->mass, p->mass + T);
    for (double m : h->mass)
      if (!(m > 0) || !std::isfinite(m)) { delete h; return fail(nullptr, NEP_ERR_ARG, "mass must be positive"); }
  }
  model_constants(h->mf);
  cudaGetDevice(&h->device);
  cudaError_t e = cudaMallocHost(&h->h_status, sizeof(BuildStatus));
  if (e != cudaSuccess) { delete h; return fail(nullptr, NEP_ERR_CUDA, "pinned alloc failed"); }
  std::memset(h->h_status, 0, sizeof(BuildStatus));
  if (h->d_cR.ensure(h->cR.size()) != cudaSuccess || h->d_cA.ensure(h->cA.size()) != cudaSuccess ||
      h->d_inv_mk.ensure(T) != cudaSuccess || h->d_mk_half.ensure(T) != cudaSuccess) {
    nep_destroy(h);
    return fail(nullptr, NEP_ERR_OOM, "device alloc failed");
  }
  std::vector<double> imk(T, 0.0), mkh(T, 0.0);
  for (int t = 0; t < T && !h->mass.empty(); ++t) {
    imk[t] = 1.0 / (h->mass[t] * kKappa);
    mkh[t] = 0.5 * h->mass[t] * kKappa;
  }
  if (h->generic) {  // the run-time-shape kernels read the network from global memory
    std::vector<float> ann(h->w0);
    ann.insert(ann.end(), h->b0.begin(), h->b0.end());
    ann.insert(ann.end(), h->w1.begin(), h->w1.end());
    ann.push_back(h->b1);
    if (h->d_ann.ensure(ann.size()) != cudaSuccess ||
        cudaMemcpy(h->d_ann.p, ann.data(), ann.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      nep_destroy(h);
      return fail(nullptr, NEP_ERR_OOM, "device alloc failed");
    }
  }
  cudaMemcpy(h->d_cR.p, h->cR.data(), h->cR.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_cA.p, h->cA.data(), h->cA.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(h->d_inv_mk.p, imk.data(), T * sizeof(double), cudaMemcpyHostToDevice);
  e = cudaMemcpy(h->d_mk_half.p, mkh.data(), T * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { nep_destroy(h); return fail(nullptr, NEP_ERR_CUDA, cudaGetErrorString(e)); }
  for (int sl = 0; sl < N_SLOTS; ++sl)
    for (int w = 0; w < 2; ++w) cudaEventCreate(&h->ev[sl][w]);
  cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking);
  *out = h;
  return NEP_OK;
}

int nep_destroy(nep_handle *h) {
  if (!h) return NEP_OK;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->fire_graph) cudaGraphExecDestroy(h->fire_graph);
  h->fire.release();
  h->ck_fire.release();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
  for (int sl = 0; sl < N_SLOTS; ++sl)
    for (int w = 0; w < 2; ++w)
      if (h->ev[sl][w]) cudaEventDestroy(h->ev[sl][w]);
  if (h->h_status) cudaFreeHost(h->h_status);
  h->d_cR.release(); h->d_cA.release(); h->d_inv_mk.release(); h->d_mk_half.release();
  h->x.release(); h->v.release(); h->F.release(); h->x_ref.release(); h->origin.release();
  h->partial_atom.release(); h->partial_gather.release(); h->thermo_stage.release();
  h->ck_x.release(); h->ck_v.release(); h->ck_F.release(); h->ck_types.release(); h->ck_perm.release();
  h->x2.release(); h->v2.release(); h->F2.release(); h->types2.release(); h->perm2.release(); h->cell2.release();
  h->perm.release();
  h->types.release(); h->cell_of.release(); h->cell_count.release(); h->cell_cursor.release();
  h->cell_start.release(); h->cell_atoms.release(); h->nn_r.release(); h->nn_a.release(); h->rev_a.release();
  h->thermo_ctl.release(); h->nl_r.release(); h->nl_a.release(); h->pos4.release(); h->dtab.release();
  h->posA.release();
  h->e_slots.release(); h->e_slots_ck.release(); h->e_energy.release(); h->e_virial.release(); h->e_u.release();
  h->e_w.release(); h->e_xck.release(); h->e_vck.release(); h->e_table.release();
  h->stage_e.release(); h->stage_g.release();
  h->p_ang.release(); h->e_rad.release(); h->status.release(); h->d_tc.release(); h->d_ann.release();
  h->d_grids.release(); h->d_sid.release(); h->d_offsets.release(); h->b_e.release(); h->b_w.release();
  if (h->b_graph) cudaGraphExecDestroy(h->b_graph);
  if (h->e_graph) cudaGraphExecDestroy(h->e_graph);
  h->pop_cr.release(); h->pop_ca.release(); h->pop_ann.release(); h->pop_tc.release(); h->pop_reg.release();
  h->pop_es.release(); h->pop_ws.release();
  delete h;
  return NEP_OK;
}

const char *nep_last_error(const nep_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int nep_n_des(const nep_handle *h) { return valid_handle(h) ? h->n_des : NEP_ERR_ARG; }

int nep_compute(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box, double *energy,
                double *energy_total, double *force, double *virial, double *virial_total, nep_stream_t stream) {
  nep::NvtxRange nvtx_range("nep_compute");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_atoms < 0 || !box) return fail(h, NEP_ERR_ARG, "n_atoms < 0 or box is null");
  if (n_atoms > 0 && (!pos || !types || !force)) return fail(h, NEP_ERR_ARG, "pos, types and force are required");
  h->md_ready = false;
  for (int sl = 0; sl < N_SLOTS; ++sl) h->slot_ran[sl] = false;
  if (n_atoms == 0) {
    if (energy_total) CK(cudaMemsetAsync(energy_total, 0, sizeof(double), s), "memset");
    if (virial_total) CK(cudaMemsetAsync(virial_total, 0, 9 * sizeof(double), s), "memset");
    return NEP_OK;
  }
  ev_record(h, SLOT_REBUILD, 0, s, false);
  int rc = load_structure(h, n_atoms, pos, types, box, s);
  if (rc) return rc;
  ev_record(h, SLOT_REBUILD, 1, s, false);
  rc = run_forces(h, n_atoms, energy, force, virial, 0, 0.0, s, false);
  if (rc) return rc;
  ev_record(h, SLOT_FINAL, 0, s, false);
  launch_finalize(h->ops->atom_blocks(n_atoms), h->partial_atom.p, h->ops->gather_blocks(n_atoms),
                  h->partial_gather.p, energy_total, virial_total, nullptr, nullptr, nullptr, n_atoms, h->volume,
                  nullptr, s);
  ev_record(h, SLOT_FINAL, 1, s, false);
  CK(cudaGetLastError(), "finalize");
  return NEP_OK;
}

int nep_compute_batch(nep_handle *h, int n_struct, const int *offsets, const double *pos, const int *types,
                      const double *boxes, double *energy, double *energy_struct, double *force, double *virial,
                      double *virial_struct, nep_stream_t stream) {
  nep::NvtxRange nvtx_range("nep_compute_batch");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_offsets(h, n_struct, offsets);
  if (rc) return rc;
  if (n_struct > 0 && !boxes) return fail(h, NEP_ERR_ARG, "boxes is null");
  const int N = n_struct > 0 ? offsets[n_struct] : 0;
  if (N > 0 && (!pos || !types || !force)) return fail(h, NEP_ERR_ARG, "pos, types and force are required");
  h->md_ready = false;
  for (int sl = 0; sl < N_SLOTS; ++sl) h->slot_ran[sl] = false;
  if (N == 0) {
    if (energy_struct && n_struct) CK(cudaMemsetAsync(energy_struct, 0, sizeof(double) * n_struct, s), "memset");
    if (virial_struct && n_struct) CK(cudaMemsetAsync(virial_struct, 0, 9 * sizeof(double) * n_struct, s), "memset");
    return NEP_OK;
  }
  rc = setup_batch(h, n_struct, offsets, boxes, N, s);
  if (rc) return rc;
  BatchOut o;
  o.pos = pos;
  o.types = types;
  o.e_atom = energy;
  o.w_atom = virial;
  o.force = force;
  o.e_struct = energy_struct;
  o.w_struct = virial_struct;
  if (!o.e_atom && energy_struct) {
    CK(h->b_e.ensure(N), "alloc");
    o.e_atom = h->b_e.p;
  }
  if (!o.w_atom && virial_struct) {
    CK(h->b_w.ensure(9 * (size_t)N), "alloc");
    o.w_atom = h->b_w.p;
  }
  // a repeated call (same layout, arrays and list capacities) replays one captured graph:
  // copy-in, neighbour build, both kernels and the structure sums, then one status read
  BatchKey key = batch_key(h, N, o);
  if (!h->prof && h->b_graph && std::memcmp(&key, &h->b_key, sizeof(key)) == 0) {
    CK(cudaGraphLaunch(h->b_graph, s), "batch graph launch");
    CK(wait_stream(s), "batch graph");
    const BuildStatus &st = *h->h_status;
    if (st.bad_input & 1) return fail(h, NEP_ERR_ARG, "atom type out of range");
    if (st.bad_input & 2) return fail(h, NEP_ERR_NONFINITE, "non-finite position");
    if (st.tc_timeout) return fail(h, NEP_ERR_TIMEOUT, "a tensor-core completion wait ran out");
    if (!st.overflow && !st.rev_missing) return NEP_OK;
    // the lists outgrew their capacity: size them again on the eager path below
  }
  ev_record(h, SLOT_REBUILD, 0, s, false);
  CK(cudaMemcpyAsync(h->x.p, pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy pos");
  CK(cudaMemcpyAsync(h->types.p, types, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "copy types");
  launch_iota(N, h->perm.p, s);
  h->N = N;
  h->stats_cache.n_atoms = N;
  for (int a = 0; a < 3; ++a) h->stats_cache.cells[a] = 0;
  rc = rebuild_lists(h, N, s, batch_of(h));
  if (rc) return rc;
  ev_record(h, SLOT_REBUILD, 1, s, false);
  rc = batch_kernels(h, N, o, s, false);
  if (rc) return rc;
  if (!h->prof) {
    key = batch_key(h, N, o);
    if (std::memcmp(&key, &h->b_last, sizeof(key)) == 0) {
      rc = capture_batch(h, N, o, s);  // the second identical call: capture for the next ones
      if (rc) return rc;
      h->b_key = key;
    }
    h->b_last = key;
  }
  return NEP_OK;
}

int nep_n_par(const nep_handle *h) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  const int T2 = h->T * h->T;
  return T2 * (h->nR + 1) * (h->KR + 1) + T2 * (h->nA + 1) * (h->KA + 1) + h->H * h->n_des + 2 * h->H + 1;
}

int nep_eval_population(nep_handle *h, int n_pop, const double *z, int n_struct, const int *offsets,
                        const double *pos, const int *types, const double *boxes, const double *e_tar,
                        const double *f_tar, const double *w_tar, const double *lambda, double *loss,
                        nep_stream_t stream) {
  nep::NvtxRange nvtx_range("nep_eval_population");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_offsets(h, n_struct, offsets);
  if (rc) return rc;
  if (n_pop < 0) return fail(h, NEP_ERR_ARG, "n_pop < 0");
  if (n_pop == 0) return NEP_OK;
  const int N = n_struct > 0 ? offsets[n_struct] : 0;
  if (N == 0) return fail(h, NEP_ERR_ARG, "the structure set holds no atoms");
  if (!z || !boxes || !pos || !types || !e_tar || !f_tar || !lambda || !loss)
    return fail(h, NEP_ERR_ARG, "z, boxes, pos, types, e_tar, f_tar, lambda and loss are required");
  for (int c = 0; c < 5; ++c)
    if (!std::isfinite(lambda[c])) return fail(h, NEP_ERR_ARG, "non-finite lambda");
  h->md_ready = false;
  for (int sl = 0; sl < N_SLOTS; ++sl) h->slot_ran[sl] = false;
  rc = setup_batch(h, n_struct, offsets, boxes, N, s);
  if (rc) return rc;
  ev_record(h, SLOT_REBUILD, 0, s, false);
  CK(cudaMemcpyAsync(h->x.p, pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy pos");
  CK(cudaMemcpyAsync(h->types.p, types, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "copy types");
  launch_iota(N, h->perm.p, s);
  h->N = N;
  h->stats_cache.n_atoms = N;
  rc = rebuild_lists(h, N, s, batch_of(h));
  if (rc) return rc;
  ev_record(h, SLOT_REBUILD, 1, s, false);
  // parameter vectors -> FP32 kernel arrays (and BF16 tiles for the tensor-core network)
  const int T2 = h->T * h->T;
  const int n_cr = T2 * (h->nR + 1) * (h->KR + 1), n_ca = T2 * (h->nA + 1) * (h->KA + 1);
  const int n_par = nep_n_par(h), n_ann = n_par - n_cr - n_ca;
  CK(h->pop_cr.ensure((size_t)n_pop * n_cr), "alloc population");
  CK(h->pop_ca.ensure((size_t)n_pop * n_ca), "alloc population");
  CK(h->pop_ann.ensure((size_t)n_pop * n_ann), "alloc population");
  CK(h->pop_reg.ensure(2 * (size_t)n_pop), "alloc population");
  launch_unpack_population(n_pop, z, n_par, n_cr, n_ca, h->pop_cr.p, h->pop_ca.p, h->pop_ann.p, h->pop_reg.p, s);
  const long long s_tc = (long long)h->ops->np1 * h->ops->kp1 * 2 * 4 / 16;  // four tiles, uint4 units
  if (h->precision >= 1) {
    CK(h->pop_tc.ensure((size_t)n_pop * s_tc), "alloc population");
    CK(cudaMemsetAsync(h->pop_tc.p, 0, sizeof(uint4) * (size_t)n_pop * s_tc, s), "memset tiles");
    launch_population_tiles(n_pop, h->pop_ann.p, n_ann, h->H, h->n_des, h->ops->kp1, h->ops->np1,
                            reinterpret_cast<unsigned short *>(h->pop_tc.p), s);
  }
  // members evaluated per launch (grid.y): the tuned value, else as many as the workspace
  // budget holds
  const int est = ((h->KR + 2) + 3) / 4 * 4;
  const double per_member = 4.0 * N * h->T * est + 16.0 * h->cap_a * N + 8.0 * N + (w_tar ? 72.0 * N : 0.0) +
                            80.0 * n_struct + 8.0 * kReduceSlots * (N / 64.0 + 2);
  int pc = h->tune.members;
  if (pc <= 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double budget = std::min(0.5 * (double)free_b, 32.0 * (1ull << 30));
    pc = (int)std::max(1.0, std::min((double)n_pop, budget / per_member));
  }
  pc = std::min(pc, n_pop);
  const int nb_g = (N + gather_block(h) - 1) / gather_block(h);
  CK(h->e_rad.ensure((size_t)pc * N * h->T * est), "alloc population");
  CK(h->p_ang.ensure((size_t)pc * h->cap_a * N), "alloc population");
  CK(h->b_e.ensure((size_t)pc * N), "alloc population");
  if (w_tar) CK(h->b_w.ensure((size_t)pc * N * 9), "alloc population");
  CK(h->pop_es.ensure((size_t)pc * n_struct), "alloc population");
  if (w_tar) CK(h->pop_ws.ensure((size_t)pc * n_struct * 9), "alloc population");
  rc = ensure_partials(h, N, pc);
  if (rc) return rc;
  for (int p0 = 0; p0 < n_pop; p0 += pc) {
    const int m = std::min(pc, n_pop - p0);
    AtomArgs a = make_args(h, N);
    a.energy = h->b_e.p;
    a.force = nullptr;
    a.virial = w_tar ? h->b_w.p : nullptr;
    a.s_out = N;
    a.c_r = h->pop_cr.p + (size_t)p0 * n_cr;
    a.s_cr = n_cr;
    a.c_a = h->pop_ca.p + (size_t)p0 * n_ca;
    a.s_ca = n_ca;
    a.pop_ann = h->pop_ann.p + (size_t)p0 * n_ann;
    a.s_ann = n_ann;
    a.pop_tc = h->precision >= 1 ? h->pop_tc.p + (size_t)p0 * s_tc : nullptr;
    a.s_tc = s_tc;
    a.s_erad = (long long)N * h->T * est;
    a.s_pang = (long long)h->cap_a * N;
    a.f_tar = f_tar;
    ev_record(h, SLOT_ATOM, 0, s, false);
    cudaError_t e = h->ops->atom_batch(a, h->mf, nullptr, nullptr, nullptr, 0.f, m, atom_block(h), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "nep_atom kernel (population)");
    ev_record(h, SLOT_ATOM, 1, s, false);
    ev_record(h, SLOT_GATHER, 0, s, false);
    e = h->ops->gather_batch(a, m, gather_block(h), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "nep_gather kernel (population)");
    ev_record(h, SLOT_GATHER, 1, s, false);
    ev_record(h, SLOT_FINAL, 0, s, false);
    launch_struct_sums(n_struct, m, h->d_offsets.p, N, h->b_e.p, w_tar ? h->b_w.p : nullptr, h->pop_es.p,
                       w_tar ? h->pop_ws.p : nullptr, max_struct_atoms(h), s);
    launch_population_loss(m, n_struct, h->d_offsets.p, h->pop_es.p, w_tar ? h->pop_ws.p : nullptr, e_tar, w_tar,
                           h->partial_gather.p, nb_g, N, h->pop_reg.p + 2 * (size_t)p0, n_par, lambda,
                           loss + 6 * (size_t)p0, s);
    ev_record(h, SLOT_FINAL, 1, s, false);
    CK(cudaGetLastError(), "population loss");
  }
  h->tune.last_members = pc;
  return NEP_OK;
}

int nep_autotune(nep_handle *h, int n_struct, const int *offsets, const double *pos, const int *types,
                 const double *boxes, int n_pop, nep_tuning *out, nep_stream_t stream) {
  nep::NvtxRange nvtx_range("nep_autotune");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_offsets(h, n_struct, offsets);
  if (rc) return rc;
  const int N = n_struct > 0 ? offsets[n_struct] : 0;
  if (N == 0 || !boxes || !pos || !types) return fail(h, NEP_ERR_ARG, "autotune needs a non-empty structure set");
  if (n_pop < 0 || n_pop > 65535) return fail(h, NEP_ERR_ARG, "n_pop must be in 0..65535");
  h->md_ready = false;
  rc = setup_batch(h, n_struct, offsets, boxes, N, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->x.p, pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy pos");
  CK(cudaMemcpyAsync(h->types.p, types, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "copy types");
  launch_iota(N, h->perm.p, s);
  h->N = N;
  rc = rebuild_lists(h, N, s, batch_of(h));
  if (rc) return rc;
  // candidates: atoms per CTA of both kernels, then (for a population) members per launch
  const int est = ((h->KR + 2) + 3) / 4 * 4;
  const double per_member = 4.0 * N * h->T * est + 16.0 * h->cap_a * N + 8.0 * N + 8.0 * kReduceSlots * (N / 64.0 + 2);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const double budget = std::min(0.5 * (double)free_b, 32.0 * (1ull << 30));
  const int max_members = std::max(1, std::min(std::max(n_pop, 1), (int)std::min(65535.0, budget / per_member)));
  CK(h->e_rad.ensure((size_t)max_members * N * h->T * est), "alloc autotune");
  CK(h->p_ang.ensure((size_t)max_members * h->cap_a * N), "alloc autotune");
  CK(h->b_e.ensure((size_t)max_members * N), "alloc autotune");
  const Tuning saved = h->tune;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time one batched evaluation (atom + gather kernels) of `m` members; best of 3 after a warm-up
  auto time_eval = [&](int m, float *ms) -> int {
    int r = ensure_partials(h, N, m);
    if (r) return r;
    AtomArgs a = make_args(h, N);
    a.energy = h->b_e.p;
    a.s_out = N;
    a.s_erad = (long long)N * h->T * est;
    a.s_pang = (long long)h->cap_a * N;
    float best = 1e30f;
    for (int it = 0; it < 4; ++it) {
      cudaEventRecord(e0, s);
      cudaError_t e = h->ops->atom_batch(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, m,
                                         atom_block(h), s);
      if (e == cudaSuccess) e = h->ops->gather_batch(a, m, gather_block(h), s);
      if (e != cudaSuccess) return cuda_fail(h, e, "autotune launch");
      cudaEventRecord(e1, s);
      CK(cudaEventSynchronize(e1), "autotune");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (it > 0) best = std::min(best, t);
    }
    *ms = best;
    return NEP_OK;
  };
  int n_tried = 0;
  float best_ms = 1e30f, default_ms = 0.f;
  int best_ab = 128, best_gb = 128;
  const int abs_[2] = {64, 128}, gbs[3] = {64, 128, 256};
  for (int ia = 0; ia < 2 && !rc; ++ia) {
    // the tensor-core forms, the run-time-shape kernels and the low-register FP32 form work on
    // 128-atom CTAs only (a 64-atom CTA would change the FP32 form, hence the rounding)
    if ((h->precision >= 1 || h->generic || atom_form_of(h) == 3) && abs_[ia] != 128) continue;
    for (int ig = 0; ig < 3 && !rc; ++ig) {
      if (h->generic && gbs[ig] != 128) continue;  // one block shape for the run-time-shape kernels
      h->tune.atom_block = abs_[ia];
      h->tune.gather_block = gbs[ig];
      float t = 0.f;
      rc = time_eval(1, &t);
      ++n_tried;
      if (abs_[ia] == 128 && gbs[ig] == 128) default_ms = t;
      if (!rc && t < best_ms) {
        best_ms = t;
        best_ab = abs_[ia];
        best_gb = gbs[ig];
      }
    }
  }
  h->tune.atom_block = best_ab;
  h->tune.gather_block = best_gb;
  int best_m = 0;
  if (!rc && n_pop > 0) {
    float best_per = best_ms;
    best_m = 1;
    for (int m = 2; m <= max_members && !rc; m *= 2) {
      float t = 0.f;
      rc = time_eval(m, &t);
      ++n_tried;
      if (!rc && t / m < best_per) {
        best_per = t / m;
        best_m = m;
      }
    }
    best_ms = best_per;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    h->tune = saved;
    return rc;
  }
  h->tune.members = best_m;
  h->tune.n_tried = n_tried;
  h->tune.best_ms = best_ms;
  h->tune.default_ms = default_ms;
  return out ? nep_get_tuning(h, out) : NEP_OK;
}

int nep_set_tuning(nep_handle *h, const nep_tuning *t) {
  if (!valid_handle(h) || !t) return NEP_ERR_ARG;
  if (t->members_per_launch < 0 || t->members_per_launch > 65535)
    return fail(h, NEP_ERR_ARG, "members_per_launch must be in 0..65535");
  if (t->atom_block != 0 && t->atom_block != 64 && t->atom_block != 128)
    return fail(h, NEP_ERR_ARG, "atom_block must be 0, 64 or 128");
  if (t->gather_block != 0 && t->gather_block != 64 && t->gather_block != 128 && t->gather_block != 256)
    return fail(h, NEP_ERR_ARG, "gather_block must be 0, 64, 128 or 256");
  if (h->generic && ((t->atom_block != 0 && t->atom_block != 128) || (t->gather_block != 0 && t->gather_block != 128)))
    return fail(h, NEP_ERR_UNSUPPORTED, "the run-time-shape kernels take 128 atoms per CTA");
  if (t->atom_form != 0 && t->atom_form != 1 && t->atom_form != 3)
    return fail(h, NEP_ERR_ARG, "atom_form must be 0, 1 or 3");
  h->tune.atom_form = t->atom_form;
  h->tune.members = t->members_per_launch;
  h->tune.atom_block = t->atom_block;
  h->tune.gather_block = t->gather_block;
  return NEP_OK;
}

int nep_get_tuning(const nep_handle *h, nep_tuning *t) {
  if (!valid_handle(h) || !t) return NEP_ERR_ARG;
  t->members_per_launch = h->tune.members;
  t->atom_block = h->tune.atom_block;
  t->gather_block = h->tune.gather_block;
  t->last_members = h->tune.last_members;
  t->n_tried = h->tune.n_tried;
  t->best_ms = h->tune.best_ms;
  t->default_ms = h->tune.default_ms;
  t->atom_form = atom_form_of(h);
  return NEP_OK;
}

int nep_descriptors(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box, double *q,
                    nep_stream_t stream) {
  nep::NvtxRange nvtx_range("nep_descriptors");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_atoms < 0 || !box) return fail(h, NEP_ERR_ARG, "n_atoms < 0 or box is null");
  if (n_atoms == 0) return NEP_OK;
  if (!pos || !types || !q) return fail(h, NEP_ERR_ARG, "null pointer");
  h->md_ready = false;
  int rc = load_structure(h, n_atoms, pos, types, box, s);
  if (rc) return rc;
  AtomArgs a = make_args(h, n_atoms);
  a.q_out = q;
  cudaError_t e = h->ops->atom(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, 1, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "descriptor kernel");
  return NEP_OK;
}

int nep_compute_host(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box, double *energy,
                     double *energy_total, double *force, double *virial, double *virial_total) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (n_atoms < 0 || !box || (n_atoms > 0 && (!pos || !types || !force)))
    return fail(h, NEP_ERR_ARG, "invalid arguments");
  const size_t N = (size_t)std::max(n_atoms, 1);
  double *dpos = nullptr, *dE = nullptr, *dF = nullptr, *dW = nullptr, *dtot = nullptr;
  int *dT = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
  al((void **)&dpos, 3 * N * sizeof(double));
  al((void **)&dT, N * sizeof(int));
  al((void **)&dF, 3 * N * sizeof(double));
  al((void **)&dtot, 10 * sizeof(double));
  if (energy) al((void **)&dE, N * sizeof(double));
  if (virial) al((void **)&dW, 9 * N * sizeof(double));
  int rc = NEP_OK;
  if (e != cudaSuccess) rc = cuda_fail(h, e, "nep_compute_host alloc");
  if (!rc && n_atoms > 0) {
    cudaMemcpy(dpos, pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice);
    e = cudaMemcpy(dT, types, N * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "copy in");
  }
  if (!rc) rc = nep_compute(h, n_atoms, dpos, dT, box, dE, dtot, dF, dW, dtot + 1, nullptr);
  if (!rc) {
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(h, e, "nep_compute_host");
  }
  if (!rc) {
    double tot[10];
    cudaMemcpy(tot, dtot, sizeof(tot), cudaMemcpyDeviceToHost);
    if (energy_total) *energy_total = tot[0];
    if (virial_total) std::memcpy(virial_total, tot + 1, 9 * sizeof(double));
    if (n_atoms > 0) {
      cudaMemcpy(force, dF, 3 * N * sizeof(double), cudaMemcpyDeviceToHost);
      if (energy) cudaMemcpy(energy, dE, N * sizeof(double), cudaMemcpyDeviceToHost);
      if (virial) cudaMemcpy(virial, dW, 9 * N * sizeof(double), cudaMemcpyDeviceToHost);
    }
  }
  cudaFree(dpos); cudaFree(dT); cudaFree(dF); cudaFree(dtot);
  if (dE) cudaFree(dE);
  if (dW) cudaFree(dW);
  return rc;
}

int md_init(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box, const double *vel,
            nep_stream_t stream) {
  nep::NvtxRange nvtx_range("md_init");
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (h->mass.empty()) return fail(h, NEP_ERR_ARG, "md_init needs params->mass");
  if (n_atoms < 1 || !pos || !types || !box) return fail(h, NEP_ERR_ARG, "md_init needs atoms, types and a box");
  h->md_ready = false;
  // velocities enter in the caller's order; the neighbour build below moves them into the
  // internal (cell) order together with positions, types and perm
  int rc = ensure_atoms(h, n_atoms, s);
  if (rc) return rc;
  if (vel) CK(cudaMemcpyAsync(h->v.p, vel, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToDevice, s), "copy vel");
  else CK(cudaMemsetAsync(h->v.p, 0, sizeof(double) * 3 * n_atoms, s), "memset vel");
  rc = load_structure(h, n_atoms, pos, types, box, s);
  if (rc) return rc;
  rc = run_forces(h, n_atoms, nullptr, h->F.p, nullptr, 0, 0.0, s, false);
  if (rc) return rc;
  CK(wait_stream(s), "md_init");
  h->h_status->n_rebuilds = 0;
  h->h_status->md_steps = 0;
  h->h_status->rebuild = 0;
  CK(cudaMemcpy(h->status.p, h->h_status, sizeof(BuildStatus), cudaMemcpyHostToDevice), "status");
  for (cudaGraphExec_t *g : {&h->graph, &h->fire_graph})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  h->md_ready = true;
  return NEP_OK;
}

int md_init_host(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                 const double *vel) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (n_atoms < 1 || !pos || !types || !box) return fail(h, NEP_ERR_ARG, "md_init needs atoms, types and a box");
  // the host arrays go straight into the handle's reorder scratch (no temporary device
  // buffers); md_init copies them on the same stream before the neighbour build reuses it
  int rc = ensure_atoms(h, n_atoms, nullptr);
  if (rc) return rc;
  const size_t b3 = sizeof(double) * 3 * (size_t)n_atoms;
  CK(cudaMemcpyAsync(h->x2.p, pos, b3, cudaMemcpyHostToDevice, nullptr), "md_init_host");
  CK(cudaMemcpyAsync(h->types2.p, types, sizeof(int) * (size_t)n_atoms, cudaMemcpyHostToDevice, nullptr),
     "md_init_host");
  if (vel) CK(cudaMemcpyAsync(h->v2.p, vel, b3, cudaMemcpyHostToDevice, nullptr), "md_init_host");
  rc = md_init(h, n_atoms, h->x2.p, h->types2.p, box, vel ? h->v2.p : nullptr, nullptr);
  if (rc) return rc;
  CK(cudaStreamSynchronize(nullptr), "md_init_host");
  return NEP_OK;
}

namespace {
// Launch one MD step on stream s (used both for capture and, if needed, directly).
// One velocity-Verlet step (with `fire`: one FIRE step, the time step read on the device).
int md_step_launch(nep_handle *h, double dt, cudaStream_t s, bool capturing, bool fire = false) {
  const int N = h->N;
  const double half_skin2 = 0.25 * h->skin * h->skin;
  FireState *fs = fire ? h->fire.p : nullptr;
  ev_record(h, SLOT_DRIFT, 0, s, capturing);
  launch_drift(N, atom_state(h), h->d_inv_mk.p, dt, half_skin2, h->status.p, s, fs);
  ev_record(h, SLOT_DRIFT, 1, s, capturing);
  ev_record(h, SLOT_REBUILD, 0, s, capturing);
  const float rlR = (float)(h->rcR + h->skin), rlA = (float)(h->rcA + h->skin);
  if (capturing && h->graph_cond) {
    // the rebuild kernels sit in the body of a conditional (IF) node; a one-thread kernel sets
    // its condition from the drift kernel's request, so steps without a rebuild launch none
    cudaStreamCaptureStatus cs;
    unsigned long long id = 0;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &edges, &nd), "capture info");
    cudaGraphConditionalHandle hc;
    CK(cudaGraphConditionalHandleCreate(&hc, g, 0, 0), "conditional handle");
    launch_rebuild_condition(hc, h->status.p, s);
    CK(cudaGetLastError(), "condition kernel");
    CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &edges, &nd), "capture info");
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, g, deps, edges, nd, &np), "conditional node");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies), "capture deps");
    CK(cudaStreamBeginCaptureToGraph(h->cap_stream2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
       "capture body");
    cudaError_t e = launch_rebuild(N, h->T, h->grid, Batch{}, h->dtab.p, rlR * rlR, rlA * rlA, h->rcR2f(), h->rcA2f(),
                                   atom_state(h), list_bufs(h), 0, h->status.p, h->cap_stream2);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream2, &out);
    if (e != cudaSuccess) return cuda_fail(h, e, "launch rebuild");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "end body capture");
    size_t nn = 0;
    cudaGraphGetNodes(body, nullptr, &nn);
    h->rebuild_kernels = (int)nn;
  } else {
    CK(launch_rebuild(N, h->T, h->grid, Batch{}, h->dtab.p, rlR * rlR, rlA * rlA, h->rcR2f(), h->rcA2f(), atom_state(h),
                      list_bufs(h), 0, h->status.p, s),
       "launch rebuild");
    h->rebuild_kernels = 0;
  }
  ev_record(h, SLOT_REBUILD, 1, s, capturing);
  int rc = run_forces(h, N, nullptr, h->F.p, nullptr, 1, 0.5 * dt, s, capturing, fs);
  if (rc) return rc;
  ev_record(h, SLOT_FINAL, 0, s, capturing);
  ThermoState *ts = (!fire && h->nvt) ? h->thermo_state.p : nullptr;
  if (ts) launch_thermostat(N, atom_state(h), h->ops->gather_blocks(N), h->partial_gather.p, ts, s);
  launch_finalize(h->ops->atom_blocks(N), h->partial_atom.p, h->ops->gather_blocks(N), h->partial_gather.p, nullptr,
                  nullptr, nullptr, h->thermo_stage.p, h->thermo_ctl.p, N, h->volume, ts, s);
  if (fire) launch_fire_mix(N, atom_state(h), fs, 0, s);
  ev_record(h, SLOT_FINAL, 1, s, capturing);
  CK(cudaGetLastError(), "md step launch");
  return NEP_OK;
}
}  // namespace

namespace {
int md_queue(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo, cudaStream_t s,
             bool fire = false, double *heat = nullptr) {
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "md_run before md_init");
  if (n_steps < 0 || !(dt_fs > 0) || !std::isfinite(dt_fs) || thermo_every < 1)
    return fail(h, NEP_ERR_ARG, "need n_steps >= 0, dt > 0, thermo_every >= 1");
  if (n_steps == 0) return NEP_OK;
  const bool rows_out = thermo || heat;
  const int rows = rows_out ? n_steps / thermo_every : 0;
  CK(h->thermo_stage.ensure((size_t)kThermoCols * (rows + 1)), "alloc thermo");
  int ctl[4] = {0, 0, rows_out ? thermo_every : (n_steps + 1), 0};
  CK(cudaMemcpyAsync(h->thermo_ctl.p, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s), "thermo ctl");
  // (re)capture the one-step graph when the step size, the profiling mode or the thermo
  // staging buffer changed
  cudaGraphExec_t &gx = fire ? h->fire_graph : h->graph;
  if (fire && gx && (h->graph_prof != h->prof || h->graph_thermo != h->thermo_stage.p ||
                     h->graph_cond_used != h->graph_cond || h->graph_prec != kernel_form(h) ||
                     h->graph_nvt != h->nvt)) {
    cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
  if (!gx || (!fire && h->graph_dt != dt_fs) || h->graph_prof != h->prof || h->graph_thermo != h->thermo_stage.p ||
      h->graph_cond_used != h->graph_cond || h->graph_prec != kernel_form(h) || h->graph_nvt != h->nvt) {
    // the MD and FIRE graphs share the capture settings: drop both when they change
    for (cudaGraphExec_t *g : {&h->graph, &h->fire_graph})
      if (*g) {
        cudaGraphExecDestroy(*g);
        *g = nullptr;
      }
    CK(wait_stream(s), "sync");
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
    int rc = md_step_launch(h, dt_fs, h->cap_stream, true, fire);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    h->graph_kernels = count_kernel_nodes(graph);
    e = cudaGraphInstantiate(&gx, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    if (!fire) h->graph_dt = dt_fs;
    h->graph_prof = h->prof;
    h->graph_thermo = h->thermo_stage.p;
    h->graph_cond_used = h->graph_cond;
    h->graph_prec = kernel_form(h);
    h->graph_nvt = h->nvt;
  }
  for (int st = 0; st < n_steps; ++st) CK(cudaGraphLaunch(gx, s), "graph launch");
  // rows of the staging area -> the caller's [rows][4] thermo and [rows][3] heat current
  if (thermo && rows > 0)
    CK(cudaMemcpy2DAsync(thermo, 4 * sizeof(double), h->thermo_stage.p, kThermoCols * sizeof(double),
                         4 * sizeof(double), rows, cudaMemcpyDeviceToDevice, s), "thermo");
  if (heat && rows > 0)
    CK(cudaMemcpy2DAsync(heat, 3 * sizeof(double), h->thermo_stage.p + 4, kThermoCols * sizeof(double),
                         3 * sizeof(double), rows, cudaMemcpyDeviceToDevice, s), "heat current");
  return NEP_OK;
}
}  // namespace

int md_status(nep_handle *h, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "no MD state");
  int rc = read_status(h, (cudaStream_t)stream);
  if (rc) return rc;
  if (h->h_status->tc_timeout) return fail(h, NEP_ERR_TIMEOUT, "a tensor-core completion wait ran out");
  if (h->h_status->overflow || h->h_status->rev_missing) {
    h->md_ready = false;
    return fail(h, NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour list overflow during md_run; call md_init again");
  }
  return NEP_OK;
}

int md_run_async(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  return md_queue(h, n_steps, dt_fs, thermo_every, thermo, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
// Velocity-Verlet (or FIRE) steps in chunks of whole thermo periods; each chunk starts from
// a checkpoint so that a list overflow during it can be undone: restore, grow the lists,
// rebuild, replay. A converged relaxation stops at the end of its chunk.
int run_steps(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo, cudaStream_t s, bool fire,
              double *heat = nullptr) {
  nep::NvtxRange nvtx_range("md_run");
  const int N = h->N;
  const size_t b = sizeof(double) * 3 * (size_t)N;
  CK(h->ck_x.ensure(3 * (size_t)N), "alloc checkpoint");
  CK(h->ck_v.ensure(3 * (size_t)N), "alloc checkpoint");
  CK(h->ck_F.ensure(3 * (size_t)N), "alloc checkpoint");
  CK(h->ck_types.ensure((size_t)N), "alloc checkpoint");
  CK(h->ck_perm.ensure((size_t)N), "alloc checkpoint");
  if (fire) CK(h->ck_fire.ensure(1), "alloc checkpoint");
  const bool nvt = !fire && h->nvt;
  if (nvt) CK(h->ck_thermo.ensure(1), "alloc checkpoint");
  const size_t bi = sizeof(int) * (size_t)N;
  // chunks of whole thermo periods; each chunk starts from a checkpoint so that a list
  // overflow during it can be undone: restore, grow the lists, rebuild, replay
  const int chunk = thermo_every >= 64 ? thermo_every : (64 / thermo_every) * thermo_every;
  int done = 0;
  while (done < n_steps) {
    const int c = std::min(chunk, n_steps - done);
    CK(cudaMemcpyAsync(h->ck_x.p, h->x.p, b, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_v.p, h->v.p, b, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_F.p, h->F.p, b, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_types.p, h->types.p, bi, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemcpyAsync(h->ck_perm.p, h->perm.p, bi, cudaMemcpyDeviceToDevice, s), "checkpoint");
    if (fire) CK(cudaMemcpyAsync(h->ck_fire.p, h->fire.p, sizeof(FireState), cudaMemcpyDeviceToDevice, s), "checkpoint");
    if (nvt)
      CK(cudaMemcpyAsync(h->ck_thermo.p, h->thermo_state.p, sizeof(ThermoState), cudaMemcpyDeviceToDevice, s),
         "checkpoint");
    int rc = read_status(h, s);
    if (rc) return rc;
    const long long steps0 = h->h_status->md_steps, rebuilds0 = h->h_status->n_rebuilds;
    for (int attempt = 0;; ++attempt) {
      double *th = thermo ? thermo + 4 * (size_t)(done / thermo_every) : nullptr;
      double *hc = heat ? heat + 3 * (size_t)(done / thermo_every) : nullptr;
      rc = md_queue(h, c, dt_fs, thermo_every, th, s, fire, hc);
      if (rc) return rc;
      rc = read_status(h, s);
      if (rc) return rc;
      const BuildStatus st = *h->h_status;
      if (!st.overflow && !st.rev_missing) break;
      if (attempt >= 2 || st.max_r > kListBuf || st.max_a > kListBuf) {
        h->md_ready = false;
        return fail(h, NEP_ERR_NEIGHBOR_OVERFLOW, "more than " + std::to_string(kListBuf) +
                                                      " neighbours within r_c + skin for one atom");
      }
      // undo the chunk and rebuild with larger lists
      CK(cudaMemcpyAsync(h->x.p, h->ck_x.p, b, cudaMemcpyDeviceToDevice, s), "restore");
      CK(cudaMemcpyAsync(h->v.p, h->ck_v.p, b, cudaMemcpyDeviceToDevice, s), "restore");
      CK(cudaMemcpyAsync(h->F.p, h->ck_F.p, b, cudaMemcpyDeviceToDevice, s), "restore");
      CK(cudaMemcpyAsync(h->types.p, h->ck_types.p, bi, cudaMemcpyDeviceToDevice, s), "restore");
      CK(cudaMemcpyAsync(h->perm.p, h->ck_perm.p, bi, cudaMemcpyDeviceToDevice, s), "restore");
      if (fire) CK(cudaMemcpyAsync(h->fire.p, h->ck_fire.p, sizeof(FireState), cudaMemcpyDeviceToDevice, s), "restore");
      if (nvt)
        CK(cudaMemcpyAsync(h->thermo_state.p, h->ck_thermo.p, sizeof(ThermoState), cudaMemcpyDeviceToDevice, s),
           "restore");
      rc = ensure_lists(h, N, round_cap(st.max_r), round_cap(st.max_a));
      if (rc) return rc;
      rc = rebuild_lists(h, N, s);
      if (rc) return rc;
      h->h_status->md_steps = steps0;
      h->h_status->n_rebuilds = rebuilds0;
      h->h_status->rebuild = 0;
      CK(cudaMemcpyAsync(h->status.p, h->h_status, sizeof(BuildStatus), cudaMemcpyHostToDevice, s), "status");
      for (cudaGraphExec_t *g : {&h->graph, &h->fire_graph})
        if (*g) {
          cudaGraphExecDestroy(*g);
          *g = nullptr;
        }
    }
    done += c;
    if (fire && done < n_steps) {
      FireState fs;
      CK(cudaMemcpyAsync(&fs, h->fire.p, sizeof(fs), cudaMemcpyDeviceToHost, s), "fire state");
      CK(wait_stream(s), "sync");
      if (fs.converged) {
        // the remaining steps would change nothing; keep the thermo rows complete
        if (thermo) {
          const int r0 = done / thermo_every, r1 = n_steps / thermo_every;
          for (int r = r0; r < r1 && r > 0; ++r)
            CK(cudaMemcpyAsync(thermo + 4 * (size_t)r, thermo + 4 * (size_t)(r0 - 1), 4 * sizeof(double),
                               cudaMemcpyDeviceToDevice, s), "thermo");
        }
        break;
      }
    }
  }
  return NEP_OK;
}
}  // namespace

extern "C" {

int md_run(nep_handle *h, int n_steps, double dt_fs, int thermo_every, double *thermo, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "md_run before md_init");
  if (n_steps < 0 || !(dt_fs > 0) || !std::isfinite(dt_fs) || thermo_every < 1)
    return fail(h, NEP_ERR_ARG, "need n_steps >= 0, dt > 0, thermo_every >= 1");
  return run_steps(h, n_steps, dt_fs, thermo_every, thermo, (cudaStream_t)stream, false);
}

int md_run_ex(nep_handle *h, int n_steps, double dt_fs, const md_options *opt, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "md_run_ex before md_init");
  if (!opt) return fail(h, NEP_ERR_ARG, "options are null");
  if (n_steps < 0 || !(dt_fs > 0) || !std::isfinite(dt_fs) || opt->thermo_every < 1)
    return fail(h, NEP_ERR_ARG, "need n_steps >= 0, dt > 0, thermo_every >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const bool nvt = opt->temperature > 0;
  if (nvt) {
    if (!(opt->tau_fs > 0) || !std::isfinite(opt->temperature) || !opt->bdp_random)
      return fail(h, NEP_ERR_ARG, "the thermostat needs tau_fs > 0 and bdp_random");
    if (h->N < 2) return fail(h, NEP_ERR_ARG, "the thermostat needs at least 2 atoms");
    CK(h->thermo_state.ensure(1), "alloc thermostat");
    ThermoState ts{};
    ts.nf = 3.0 * h->N - 3.0;
    ts.c = std::exp(-dt_fs / opt->tau_fs);
    ts.kbar = 0.5 * ts.nf * 8.617333262e-5 * opt->temperature;
    ts.alpha = 1.0;
    ts.rand = opt->bdp_random;
    ts.step = 0;
    CK(cudaMemcpyAsync(h->thermo_state.p, &ts, sizeof(ts), cudaMemcpyHostToDevice, s), "thermostat");
    // the host copy must outlive the asynchronous copy
    CK(wait_stream(s), "sync");
  }
  h->nvt = nvt;
  const int rc = run_steps(h, n_steps, dt_fs, opt->thermo_every, opt->thermo, s, false, opt->heat_current);
  h->nvt = false;
  return rc;
}

int nep_heat_current(nep_handle *h, int n_atoms, const double *pos, const int *types, const double *box,
                     const double *vel, double *heat, double *heat_total, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  if (n_atoms < 1 || !pos || !types || !box || !vel || (!heat && !heat_total))
    return fail(h, NEP_ERR_ARG, "need atoms, velocities and an output");
  cudaStream_t s = (cudaStream_t)stream;
  h->md_ready = false;
  int rc = load_structure(h, n_atoms, pos, types, box, s);
  if (rc) return rc;
  AtomArgs a = make_args(h, n_atoms);
  a.vel_in = vel;
  a.heat = heat;
  cudaError_t e = h->ops->atom(a, h->mf, h->w0.data(), h->b0.data(), h->w1.data(), h->b1, 0, s);
  if (e == cudaSuccess) e = h->ops->gather(a, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "heat current kernels");
  launch_finalize(h->ops->atom_blocks(n_atoms), h->partial_atom.p, h->ops->gather_blocks(n_atoms),
                  h->partial_gather.p, nullptr, nullptr, heat_total, nullptr, nullptr, n_atoms, h->volume, nullptr,
                  s);
  CK(cudaGetLastError(), "heat current");
  return NEP_OK;
}

int fire_run(nep_handle *h, int n_steps, double dt0_fs, double fmax, double *thermo, int *steps_taken,
             nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "fire_run before md_init");
  if (n_steps < 0 || !(dt0_fs > 0) || !std::isfinite(dt0_fs) || !(fmax >= 0) || !std::isfinite(fmax))
    return fail(h, NEP_ERR_ARG, "need n_steps >= 0, dt0 > 0, fmax >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->N;
  CK(h->fire.ensure(1), "alloc fire");
  FireState fs{};
  fs.dt = dt0_fs;
  fs.alpha = 0.1;
  fs.dt_max = 10.0 * dt0_fs;
  fs.fmax2 = fmax * fmax;
  CK(cudaMemsetAsync(h->v.p, 0, sizeof(double) * 3 * (size_t)N, s), "zero velocities");
  CK(cudaMemcpyAsync(h->fire.p, &fs, sizeof(fs), cudaMemcpyHostToDevice, s), "fire state");
  launch_fire_mix(N, atom_state(h), h->fire.p, 1, s);  // already converged at the start?
  CK(cudaGetLastError(), "fire start");
  int rc = run_steps(h, n_steps, dt0_fs, 1, thermo, s, true);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&fs, h->fire.p, sizeof(fs), cudaMemcpyDeviceToHost, s), "fire state");
  CK(wait_stream(s), "sync");
  if (steps_taken) *steps_taken = fs.steps;
  return NEP_OK;
}

int md_get_state(nep_handle *h, double *pos, double *vel, double *force, nep_stream_t stream) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "no MD state");
  cudaStream_t s = (cudaStream_t)stream;
  launch_export(h->N, atom_state(h), h->grid, Batch{}, pos, vel, force, s);
  CK(cudaGetLastError(), "export");
  return NEP_OK;
}

int md_get_state_host(nep_handle *h, double *pos, double *vel, double *force) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (!h->md_ready) return fail(h, NEP_ERR_STATE, "no MD state");
  // exported into the handle's reorder scratch (idle between steps), then copied out
  const size_t b = sizeof(double) * 3 * (size_t)h->N;
  int rc = md_get_state(h, pos ? h->x2.p : nullptr, vel ? h->v2.p : nullptr, force ? h->F2.p : nullptr, nullptr);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (pos) e = cudaMemcpyAsync(pos, h->x2.p, b, cudaMemcpyDeviceToHost, nullptr);
  if (e == cudaSuccess && vel) e = cudaMemcpyAsync(vel, h->v2.p, b, cudaMemcpyDeviceToHost, nullptr);
  if (e == cudaSuccess && force) e = cudaMemcpyAsync(force, h->F2.p, b, cudaMemcpyDeviceToHost, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) return cuda_fail(h, e, "md_get_state_host");
  return NEP_OK;
}

int nep_export_lists(nep_handle *h, int cap, int *nn_r, int *j_r, float *d_r, int *nn_a, int *j_a, float *d_a) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->err.clear();
  if (cap < 1 || !nn_r || !j_r || !d_r || !nn_a || !j_a || !d_a)
    return fail(h, NEP_ERR_ARG, "cap >= 1 and every output are required");
  if (h->N <= 0 || !h->nl_r.p || !h->nl_a.p || h->cap_r <= 0 || h->cap_a <= 0)
    return fail(h, NEP_ERR_STATE, "no neighbour lists have been built");
  const int N = h->N;
  CK(cudaDeviceSynchronize(), "synchronise");
  CK(cudaMemcpy(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost), "status");
  if (h->h_status->max_r > cap || h->h_status->max_a > cap)
    return fail(h, NEP_ERR_ARG, "cap is below the longest list (nep_get_stats max_radial / max_angular)");
  const size_t rows = (size_t)N * cap;
  int *di = nullptr;
  float *df = nullptr;
  CK(cudaMalloc(&di, sizeof(int) * (2 * (size_t)N + 2 * rows)), "alloc");
  cudaError_t e = cudaMalloc(&df, sizeof(float) * 6 * rows);
  if (e != cudaSuccess) {
    cudaFree(di);
    return cuda_fail(h, e, "alloc");
  }
  int *dnr = di, *dna = di + N, *djr = di + 2 * (size_t)N, *dja = djr + rows;
  float *ddr = df, *dda = df + 3 * rows;
  launch_export_lists(N, h->T, h->pos4.p, h->perm.p, list_bufs(h), h->dtab.p, h->grid.ncode, h->grid.jbits,
                      h->grid.jmask, cap, dnr, djr, ddr, dna, dja, dda, 0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(nn_r, dnr, sizeof(int) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(nn_a, dna, sizeof(int) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(j_r, djr, sizeof(int) * rows, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(j_a, dja, sizeof(int) * rows, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d_r, ddr, sizeof(float) * 3 * rows, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d_a, dda, sizeof(float) * 3 * rows, cudaMemcpyDeviceToHost);
  cudaFree(di);
  cudaFree(df);
  if (e != cudaSuccess) return cuda_fail(h, e, "nep_export_lists");
  return NEP_OK;
}

int nep_get_stats(nep_handle *h, nep_stats *out) {
  if (!valid_handle(h) || !out) return NEP_ERR_ARG;
  nep_stats s = h->stats_cache;
  s.cap_radial = h->cap_r;
  s.cap_angular = h->cap_a;
  s.graph_kernels = h->graph_kernels;
  s.rebuild_kernels = h->rebuild_kernels;
  s.batch_graph_kernels = h->b_graph ? h->b_graph_kernels : 0;
  if (h->status.p) {
    cudaMemcpy(h->h_status, h->status.p, sizeof(BuildStatus), cudaMemcpyDeviceToHost);
    s.n_rebuilds = h->h_status->n_rebuilds;
    s.md_steps = h->h_status->md_steps;
    s.max_radial = h->h_status->max_r;
    s.max_angular = h->h_status->max_a;
    if (h->N > 0) {
      s.mean_radial = (double)h->h_status->sum_r / h->N;
      s.mean_angular = (double)h->h_status->sum_a / h->N;
    }
  }
  *out = s;
  return NEP_OK;
}

int nep_set_profiling(nep_handle *h, int enable) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->prof = enable != 0;
  return NEP_OK;
}

// BF16 (round to nearest even) of a float, as raw bits.
static uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

static float from_bf16(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

int nep_set_precision(nep_handle *h, int mode) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  if (mode < 0 || mode > 2)
    return fail(h, NEP_ERR_ARG, "precision must be 0 (FP32), 1 (BF16 tensor cores) or 2 (split BF16)");
  if (mode >= 1 && h->generic)
    return fail(h, NEP_ERR_UNSUPPORTED, "the tensor-core forms need a compiled hyper-parameter shape");
  if (mode >= 1 && !h->d_tc.p) {
    // W0 as the two GEMM operands, K-major no-swizzle UMMA layout, zero padded:
    //   B1 [NP1 x KP1]: (mu, nu) -> w0[mu][nu];  B2 [KP1 x NP1]: (nu, mu) -> w0[mu][nu]
    // first rounded to BF16, then (for the split form) the BF16 of the remainder
    const int KP1 = h->ops->kp1, NP1 = h->ops->np1, D = h->n_des, H = h->H;
    const size_t tile = (size_t)NP1 * KP1;
    std::vector<uint16_t> t(4 * tile, 0);
    auto off = [](int r, int k, int KC) { return ((r / 8) * KC + k / 8) * 64 + (r % 8) * 8 + (k % 8); };
    uint16_t *b1 = t.data(), *b2 = b1 + tile, *b1lo = b2 + tile, *b2lo = b1lo + tile;
    for (int mu = 0; mu < H; ++mu)
      for (int nu = 0; nu < D; ++nu) {
        const float x = h->w0[(size_t)mu * D + nu];
        const uint16_t v = to_bf16(x);
        const uint16_t vl = to_bf16(x - from_bf16(v));
        b1[off(mu, nu, KP1 / 8)] = v;
        b2[off(nu, mu, NP1 / 8)] = v;
        b1lo[off(mu, nu, KP1 / 8)] = vl;
        b2lo[off(nu, mu, NP1 / 8)] = vl;
      }
    CK(h->d_tc.ensure(t.size() * 2 / 16), "alloc tiles");
    CK(cudaMemcpy(h->d_tc.p, t.data(), t.size() * 2, cudaMemcpyHostToDevice), "copy tiles");
  }
  h->precision = mode;
  return NEP_OK;
}

int nep_set_graph_conditional(nep_handle *h, int enable) {
  if (!valid_handle(h)) return NEP_ERR_ARG;
  h->graph_cond = enable != 0;
  return NEP_OK;
}

int nep_kernel_slots(void) { return N_SLOTS; }

const char *nep_kernel_name(int slot) { return (slot >= 0 && slot < N_SLOTS) ? kSlotNames[slot] : ""; }

int nep_kernel_times(nep_handle *h, float *ms_out, int n_slots) {
  if (!valid_handle(h) || !ms_out) return NEP_ERR_ARG;
  for (int sl = 0; sl < n_slots && sl < N_SLOTS; ++sl) {
    ms_out[sl] = 0.f;
    if (!h->prof || !h->slot_ran[sl]) continue;
    if (cudaEventSynchronize(h->ev[sl][1]) != cudaSuccess) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[sl][0], h->ev[sl][1]) == cudaSuccess) ms_out[sl] = ms;
  }
  return NEP_OK;
}

}  // extern "C"
