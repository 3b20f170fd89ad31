// nep_descriptors_static: descriptor evaluation that allocates no device memory.
//
// Some callers cannot allocate device memory themselves or through the library (for
// example code running where cudaMalloc is forbidden or must not be called mid-run,
// such as a host program that pre-plans every allocation). For them this entry point runs
// the same neighbour build and descriptor kernels as nep_descriptors, but takes every
// scratch array (cell lists, neighbour lists, reordered atoms, model tables) from one
// file-scope device array of fixed size, resolved once per device.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/nep.h"
#include "nep_internal.cuh"

namespace nep {
int check_params(const nep_params *p, const ShapeOps **ops_out, const char **err);
int n_des_of(const nep_params *p);
void set_shape_args(AtomArgs &a, const nep_params &p, const float *ann);
void set_create_error(const char *msg);  // read back by nep_last_error(NULL)
}

using namespace nep;

namespace {

// the documented limits of include/nep.h are the real ones
constexpr size_t kStaticBytes = (size_t)NEP_STATIC_SCRATCH_BYTES;
constexpr int kStaticMaxAtoms = NEP_STATIC_MAX_ATOMS;
static_assert(kStaticBytes == ((size_t)16 << 20) && kStaticMaxAtoms == 4096,
              "the error messages below quote these limits");
constexpr int kMaxDevices = 64;

// The scratch arena. Every GPU that loads the library holds it until the process exits.
// In host code this name is only a stand-in for the device symbol: the device address comes
// from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_nep_static_scratch[kStaticBytes];

std::mutex g_mu;
void *g_base[kMaxDevices] = {};

int fail_static(int code, const char *msg) {
  set_create_error(msg);
  return code;
}

// Device address of the arena on the current device, looked up once per device.
int scratch_base(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_static(NEP_ERR_CUDA, "no usable current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_nep_static_scratch);
    if (e != cudaSuccess || !p) return fail_static(NEP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    g_base[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_base[dev]);
  return NEP_OK;
}

// Bump allocation inside the arena (256-byte aligned pieces).
struct Bump {
  unsigned char *p;
  size_t left;
  template <class T>
  T *take(size_t n) {
    const size_t b = (n * sizeof(T) + 255) & ~(size_t)255;
    if (b > left) return nullptr;
    T *r = reinterpret_cast<T *>(p);
    p += b;
    left -= b;
    return r;
  }
};

int cuda_err(cudaError_t e, const char *where) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail_static(e == cudaErrorMemoryAllocation ? NEP_ERR_OOM : NEP_ERR_CUDA, buf);
}

#define SK(call, where)                               \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_err(e_, where); \
  } while (0)

int run_build(int N, int T, const Grid &g, const float4 *dtab, float rlR2, float rlA2, float rcR2, float rcA2,
              const AtomState &a, const ListBufs &L, int count_only, BuildStatus *st_dev, BuildStatus *st_host,
              cudaStream_t s) {
  std::memset(st_host, 0, sizeof(BuildStatus));
  st_host->rebuild = 1;
  SK(cudaMemcpyAsync(st_dev, st_host, sizeof(BuildStatus), cudaMemcpyHostToDevice, s), "status");
  SK(launch_rebuild(N, T, g, Batch{}, dtab, rlR2, rlA2, rcR2, rcA2, a, L, count_only, st_dev, s), "neighbour build");
  SK(cudaMemcpyAsync(st_host, st_dev, sizeof(BuildStatus), cudaMemcpyDeviceToHost, s), "status");
  SK(cudaStreamSynchronize(s), "synchronise");
  if (st_host->bad_input & 1) return fail_static(NEP_ERR_ARG, "atom type out of range");
  if (st_host->bad_input & 2) return fail_static(NEP_ERR_NONFINITE, "non-finite position");
  return NEP_OK;
}

}  // namespace

extern "C" {

int nep_descriptors_static(const nep_params *params, int n_atoms, const double *pos, const int *types,
                           const double *box, double *q, nep_stream_t stream) {
  const ShapeOps *ops = nullptr;
  const char *perr = nullptr;
  int rc = check_params(params, &ops, &perr);
  if (rc) return fail_static(rc, perr);
  if (n_atoms < 0 || !box) return fail_static(NEP_ERR_ARG, "n_atoms < 0 or box is null");
  if (n_atoms == 0) return NEP_OK;
  if (n_atoms > kStaticMaxAtoms)
    return fail_static(NEP_ERR_ARG, "n_atoms exceeds NEP_STATIC_MAX_ATOMS (4096) of the static scratch");
  if (!pos || !types || !q) return fail_static(NEP_ERR_ARG, "pos, types and q are required");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = n_atoms, T = params->n_types;
  const int nR = params->n_max_radial, KR = params->basis_radial, nA = params->n_max_angular,
            KA = params->basis_angular, H = params->n_neuron, D = n_des_of(params);
  const double skin = params->skin > 0 ? params->skin : 1.0;

  // host-side model tables (fixed-size, on the stack)
  constexpr int kMaxW = 8192, kMaxC = 8192;
  static_assert(kMaxC >= kMaxTypes * kMaxTypes * 121, "radial table bound");
  float w0[kMaxW], b0[512], w1[512], cR[kMaxC], cA[kMaxC];
  const int ncR = T * T * (nR + 1) * (KR + 1), ncA = T * T * (nA + 1) * (KA + 1);
  if (H * D > kMaxW || H > 512 || ncR > kMaxC || ncA > kMaxC)
    return fail_static(NEP_ERR_UNSUPPORTED, "model too large for the static entry point");
  for (int v = 0; v < H * D; ++v) w0[v] = (float)params->w0[v];
  for (int v = 0; v < H; ++v) {
    b0[v] = (float)params->b0[v];
    w1[v] = (float)params->w1[v];
  }
  for (int v = 0; v < ncR; ++v) cR[v] = (float)params->c_radial[v];
  for (int v = 0; v < ncA; ++v) cA[v] = (float)params->c_angular[v];
  ModelF mf;
  model_constants(mf);

  Grid g;
  float4 dtab_h[512];
  double volume = 0;
  const char *gerr = nullptr;
  rc = build_grid(box, params->rc_radial + skin, N, g, dtab_h, &volume, &gerr);
  if (rc) return fail_static(rc, gerr);

  unsigned char *base = nullptr;
  rc = scratch_base(&base);
  if (rc) return rc;
  Bump arena{base, kStaticBytes};
  BuildStatus *st = arena.take<BuildStatus>(1);
  float4 *dtab = arena.take<float4>(g.ncode);
  float *dcR = arena.take<float>(ncR), *dcA = arena.take<float>(ncA);
  AtomState a;
  a.x = arena.take<double>(3 * (size_t)N);
  a.v = arena.take<double>(3 * (size_t)N);
  a.F = arena.take<double>(3 * (size_t)N);
  a.x_ref = arena.take<double>(3 * (size_t)N);
  a.origin = arena.take<double>(3 * (size_t)N);
  a.x2 = arena.take<double>(3 * (size_t)N);
  a.v2 = arena.take<double>(3 * (size_t)N);
  a.F2 = arena.take<double>(3 * (size_t)N);
  a.types = arena.take<int>(N);
  a.perm = arena.take<int>(N);
  a.cell_of = arena.take<int>(N);
  a.types2 = arena.take<int>(N);
  a.perm2 = arena.take<int>(N);
  a.cell2 = arena.take<int>(N);
  a.pos4 = arena.take<float4>(N);
  a.posA = arena.take<float4>(N);
  ListBufs L;
  std::memset(&L, 0, sizeof(L));
  L.cell_count = arena.take<int>(g.ncell + 1);
  L.cell_cursor = arena.take<int>(g.ncell + 1);
  L.cell_start = arena.take<int>(g.ncell + 1);
  L.cell_atoms = arena.take<int>(N);
  L.nn_r = arena.take<int>((size_t)T * N);
  L.nn_a = arena.take<int>(N);
  if (!st || !dtab || !dcR || !dcA || !a.x || !a.v || !a.F || !a.x_ref || !a.origin || !a.x2 || !a.v2 || !a.F2 ||
      !a.types || !a.perm || !a.cell_of || !a.types2 || !a.perm2 || !a.cell2 || !a.pos4 || !a.posA || !L.cell_count ||
      !L.cell_cursor || !L.cell_start || !L.cell_atoms || !L.nn_r || !L.nn_a)
    return fail_static(NEP_ERR_ARG, "structure too large for the static scratch (NEP_STATIC_SCRATCH_BYTES)");

  // inputs into the arena; the arena keeps the previous call's contents, so everything the
  // kernels read is written here first (the builder clears the cell counters itself)
  SK(cudaMemcpyAsync(dtab, dtab_h, sizeof(float4) * g.ncode, cudaMemcpyHostToDevice, s), "copy");
  SK(cudaMemcpyAsync(dcR, cR, sizeof(float) * ncR, cudaMemcpyHostToDevice, s), "copy");
  SK(cudaMemcpyAsync(dcA, cA, sizeof(float) * ncA, cudaMemcpyHostToDevice, s), "copy");
  SK(cudaMemcpyAsync(a.x, pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy pos");
  SK(cudaMemcpyAsync(a.types, types, sizeof(int) * N, cudaMemcpyDeviceToDevice, s), "copy types");
  SK(cudaMemsetAsync(a.v, 0, sizeof(double) * 3 * N, s), "clear");
  SK(cudaMemsetAsync(a.F, 0, sizeof(double) * 3 * N, s), "clear");
  launch_iota(N, a.perm, s);
  SK(cudaGetLastError(), "iota");

  const float rlR = (float)(params->rc_radial + skin), rlA = (float)(params->rc_angular + skin);
  const float rcR = (float)params->rc_radial, rcA = (float)params->rc_angular;
  BuildStatus host_st;
  // sizing pass, then the lists
  rc = run_build(N, T, g, dtab, rlR * rlR, rlA * rlA, rcR * rcR, rcA * rcA, a, L, 1, st, &host_st, s);
  if (rc) return rc;
  // the same per-atom list limit, with the same error, as the handle-based entry points
  if (host_st.max_r > kListBuf || host_st.max_a > kListBuf)
    return fail_static(NEP_ERR_NEIGHBOR_OVERFLOW, "more than 512 neighbours within r_c + skin for one atom");
  L.cap_r = host_st.max_r > 0 ? host_st.max_r : 1;
  L.cap_a = host_st.max_a > 0 ? host_st.max_a : 1;
  L.nl_r = arena.take<unsigned>((size_t)L.cap_r * N);
  L.nl_a = arena.take<unsigned>((size_t)L.cap_a * N);
  L.rev_a = arena.take<int>((size_t)L.cap_a * N);
  if (!L.nl_r || !L.nl_a || !L.rev_a)
    return fail_static(NEP_ERR_ARG, "neighbour lists too large for the static scratch (NEP_STATIC_SCRATCH_BYTES)");
  rc = run_build(N, T, g, dtab, rlR * rlR, rlA * rlA, rcR * rcR, rcA * rcA, a, L, 0, st, &host_st, s);
  if (rc) return rc;
  if (host_st.overflow || host_st.rev_missing) return fail_static(NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour build failed");

  AtomArgs args;
  std::memset(&args, 0, sizeof(args));
  args.N = N;
  args.T = T;
  args.jbits = g.jbits;
  args.jmask = g.jmask;
  args.ncode = g.ncode;
  args.rcR = rcR;
  args.rcA = rcA;
  args.pos4 = a.pos4;
  args.dtab = dtab;
  args.nl_r = L.nl_r;
  args.nn_r = L.nn_r;
  args.nl_a = L.nl_a;
  args.nn_a = L.nn_a;
  args.rev_a = L.rev_a;
  args.cap_r = L.cap_r;
  args.cap_a = L.cap_a;
  args.c_r = dcR;
  args.c_a = dcA;
  args.perm = a.perm;
  args.q_out = q;
  set_shape_args(args, *params, nullptr);  // the descriptor pass reads no network
  const cudaError_t e = ops->atom(args, mf, w0, b0, w1, (float)params->b1, 1, s);
  if (e != cudaSuccess) return cuda_err(e, "descriptor kernel");
  return NEP_OK;
}

}  // extern "C"
