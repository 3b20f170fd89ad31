// Neighbour-list construction, velocity-Verlet drift and reductions for libnep.
//
// The paper takes its neighbour lists as given (Appendix B lists NN_i^R, NN_i^A, NL_im^R,
// NL_im^A); here they are built on the GPU from a cell list:
//   bin_atoms     wrap positions into the cell (FP64), assign each atom to a grid cell,
//                 write cell-local FP32 coordinates, count atoms per cell;
//   scan_cells    exclusive prefix sum of the cell counts (one block, deterministic);
//   scatter_atoms place atoms into their cells; sort_cells orders each cell by atom index
//                 so the lists do not depend on atomic ordering;
//   build_lists   per atom: scan the (2R+1)^3 neighbouring cells (all periodic images when
//                 the cell is thin), keep pairs within r_c + skin, group the radial list by
//                 neighbour type and sort every list by distance (valid pairs first, which
//                 keeps warps convergent when the pair loops skip r >= r_c);
//   build_rev     for every angular pair (i, j, image), the slot of (j, i, -image) in the
//                 list of j, so forces are gathered without atomics (Algorithm 4's "index
//                 manipulations").
// Every builder returns early unless a rebuild is pending, so the whole sequence can sit
// in the captured MD step graph and only run when an atom moved more than skin/2.
#include "nep_internal.cuh"

namespace nep {

__device__ __forceinline__ bool rebuild_pending(const BuildStatus *st) {
  return *(volatile const int *)&st->rebuild != 0;
}

__global__ void zero_cells_kernel(int ncell, int *count, int *cursor, BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // per-build sums (the maxima are kept over the run)
    st->sum_r = st->sum_a = 0ull;
    st->in_r = st->in_a = 0ull;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    count[c] = 0;
    cursor[c] = 0;
  }
}

__global__ void bin_atoms_kernel(int N, int T, double *x, double *x_ref, double *origin, const int *types,
                                 float4 *pos4, int *cell_of, int *count, const Grid g, BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double r[3] = {x[3 * (size_t)i], x[3 * (size_t)i + 1], x[3 * (size_t)i + 2]};
  int ti = types[i];
  if (ti < 0 || ti >= T) {
    atomicOr(&st->bad_input, 1);
    ti = 0;
  }
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2])) {
    atomicOr(&st->bad_input, 2);
    r[0] = r[1] = r[2] = 0.0;
  }
  double s[3];
  int c[3];
  for (int b = 0; b < 3; ++b) {
    s[b] = r[0] * g.Hinv[0][b] + r[1] * g.Hinv[1][b] + r[2] * g.Hinv[2][b];
    s[b] -= floor(s[b]);
    int cb = (int)(s[b] * g.nc[b]);
    c[b] = cb < 0 ? 0 : (cb >= g.nc[b] ? g.nc[b] - 1 : cb);
  }
  double o[3];
  for (int b = 0; b < 3; ++b) {
    r[b] = s[0] * g.H[0][b] + s[1] * g.H[1][b] + s[2] * g.H[2][b];
    o[b] = c[0] * g.Hc[0][b] + c[1] * g.Hc[1][b] + c[2] * g.Hc[2][b];
  }
  for (int b = 0; b < 3; ++b) {
    x[3 * (size_t)i + b] = r[b];
    x_ref[3 * (size_t)i + b] = r[b];
    origin[3 * (size_t)i + b] = o[b];
  }
  pos4[i] = make_float4((float)(r[0] - o[0]), (float)(r[1] - o[1]), (float)(r[2] - o[2]), __int_as_float(ti));
  const int id = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  cell_of[i] = id;
  atomicAdd(count + id, 1);
}

// Exclusive scan of count[0..ncell) into start[0..ncell]; one block of 1024 threads.
__global__ void scan_cells_kernel(int ncell, const int *count, int *start, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  __shared__ int part[1024];
  const int per = (ncell + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  const int b1 = min(ncell, b0 + per);
  int s = 0;
  for (int c = b0; c < b1; ++c) s += count[c];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int c = b0; c < b1; ++c) {
    start[c] = run;
    run += count[c];
  }
  if (threadIdx.x == blockDim.x - 1) start[ncell] = part[threadIdx.x];
}

__global__ void scatter_atoms_kernel(int N, const int *cell_of, const int *start, int *cursor, int *cell_atoms,
                                     const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = cell_of[i];
  cell_atoms[start[c] + atomicAdd(cursor + c, 1)] = i;
}

__global__ void sort_cells_kernel(int ncell, const int *start, int *cell_atoms, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int b = start[c], e = start[c + 1];
  for (int p = b + 1; p < e; ++p) {
    const int v = cell_atoms[p];
    int q = p - 1;
    while (q >= b && cell_atoms[q] > v) {
      cell_atoms[q + 1] = cell_atoms[q];
      --q;
    }
    cell_atoms[q + 1] = v;
  }
}

// Sort key for list candidates: (group, squared distance, packed entry), ascending.
__device__ __forceinline__ bool cand_less(int ga, float ra, unsigned ea, int gb, float rb, unsigned eb) {
  if (ga != gb) return ga < gb;
  if (ra != rb) return ra < rb;
  return ea < eb;
}

// count_only: write no entries, only the length statistics (used to size the lists).
__global__ void build_lists_kernel(int N, const float4 *pos4, const int *cell_of, const int *start,
                                   const int *cell_atoms, const Grid g, const float4 *dtab, float rlR2, float rlA2,
                                   float rcR2, float rcA2, int T, int cap_r, int cap_a, int count_only,
                                   unsigned *nl_r, int *nn_r, unsigned *nl_a, int *nn_a, BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  unsigned er[kListBuf];
  float rr[kListBuf];
  unsigned char tr[kListBuf];
  unsigned ea[kListBuf];
  float ra[kListBuf];
  int nr = 0, nA = 0, inr = 0, ina = 0;
  const float4 pi = pos4[i];
  const int id = cell_of[i];
  const int cx = id / (g.nc[1] * g.nc[2]);
  const int cy = (id / g.nc[2]) % g.nc[1];
  const int cz = id % g.nc[2];
  for (int ox = -g.R[0]; ox <= g.R[0]; ++ox) {
    int x = (cx + ox) % g.nc[0];
    if (x < 0) x += g.nc[0];
    for (int oy = -g.R[1]; oy <= g.R[1]; ++oy) {
      int y = (cy + oy) % g.nc[1];
      if (y < 0) y += g.nc[1];
      for (int oz = -g.R[2]; oz <= g.R[2]; ++oz) {
        int z = (cz + oz) % g.nc[2];
        if (z < 0) z += g.nc[2];
        const unsigned code = (unsigned)(ox + g.R[0]) | ((unsigned)(oy + g.R[1]) << g.obits) |
                              ((unsigned)(oz + g.R[2]) << (2 * g.obits));
        const float4 D = dtab[code];
        const int cell = (x * g.nc[1] + y) * g.nc[2] + z;
        const bool self_image = (ox == 0 && oy == 0 && oz == 0);
        for (int p = start[cell]; p < start[cell + 1]; ++p) {
          const int j = cell_atoms[p];
          if (self_image && j == i) continue;
          const float4 pj = pos4[j];
          const float r2 = norm2(pair_vector(pi, pj, D));
          const unsigned ent = (unsigned)j | (code << g.jbits);
          inr += r2 < rcR2;
          ina += r2 < rcA2;
          if (r2 < rlR2) {
            if (nr < kListBuf) {
              er[nr] = ent;
              rr[nr] = r2;
              tr[nr] = (unsigned char)type_of(pj);
            }
            ++nr;
          }
          if (r2 < rlA2) {
            if (nA < kListBuf) {
              ea[nA] = ent;
              ra[nA] = r2;
            }
            ++nA;
          }
        }
      }
    }
  }
  atomicMax(&st->max_r, nr);
  atomicMax(&st->max_a, nA);
  atomicAdd(&st->sum_r, (unsigned long long)nr);
  atomicAdd(&st->sum_a, (unsigned long long)nA);
  atomicAdd(&st->in_r, (unsigned long long)inr);
  atomicAdd(&st->in_a, (unsigned long long)ina);
  if (count_only) return;
  if (nr > cap_r || nA > cap_a || nr > kListBuf || nA > kListBuf) atomicOr(&st->overflow, 1);
  const int wr = min(min(nr, cap_r), kListBuf);
  const int wa = min(min(nA, cap_a), kListBuf);
  // insertion sorts: radial by (type, r2, entry), angular by (r2, entry)
  for (int p = 1; p < wr; ++p) {
    const unsigned e = er[p];
    const float r = rr[p];
    const unsigned char t = tr[p];
    int q = p - 1;
    while (q >= 0 && cand_less(t, r, e, tr[q], rr[q], er[q])) {
      er[q + 1] = er[q];
      rr[q + 1] = rr[q];
      tr[q + 1] = tr[q];
      --q;
    }
    er[q + 1] = e;
    rr[q + 1] = r;
    tr[q + 1] = t;
  }
  for (int p = 1; p < wa; ++p) {
    const unsigned e = ea[p];
    const float r = ra[p];
    int q = p - 1;
    while (q >= 0 && cand_less(0, r, e, 0, ra[q], ea[q])) {
      ea[q + 1] = ea[q];
      ra[q + 1] = ra[q];
      --q;
    }
    ea[q + 1] = e;
    ra[q + 1] = r;
  }
  for (int t = 0; t < T; ++t) nn_r[t * N + i] = 0;
  for (int p = 0; p < wr; ++p) {
    nl_r[(size_t)p * N + i] = er[p];
    nn_r[tr[p] * N + i] += 1;
  }
  for (int p = 0; p < wa; ++p) nl_a[(size_t)p * N + i] = ea[p];
  nn_a[i] = wa;
}

__global__ void build_rev_kernel(int N, const unsigned *nl_a, const int *nn_a, const Grid g, int *rev_a,
                                 BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned om = (1u << g.obits) - 1u;
  const int na = nn_a[i];
  for (int m = 0; m < na; ++m) {
    const size_t slot = (size_t)m * N + i;
    const unsigned e = nl_a[slot];
    const int j = e & g.jmask;
    const unsigned code = e >> g.jbits;
    const unsigned cx = code & om, cy = (code >> g.obits) & om, cz = (code >> (2 * g.obits)) & om;
    const unsigned rc = (2u * g.R[0] - cx) | ((2u * g.R[1] - cy) << g.obits) | ((2u * g.R[2] - cz) << (2 * g.obits));
    const unsigned target = (unsigned)i | (rc << g.jbits);
    const int nj = nn_a[j];
    int found = -1;
    for (int q = 0; q < nj; ++q)
      if (nl_a[(size_t)q * N + j] == target) {
        found = q;
        break;
      }
    if (found < 0) {
      atomicAdd(&st->rev_missing, 1);
      rev_a[slot] = (int)slot;  // points at a finite entry; the status reports the error
    } else {
      rev_a[slot] = (int)((size_t)found * N + j);
    }
  }
}

__global__ void finish_build_kernel(BuildStatus *st) {
  if (st->rebuild) {
    st->rebuild = 0;
    st->n_rebuilds += 1;
  }
}

// Velocity Verlet, first half: v += dt/2 F/m; x += dt v; refresh cell-local coordinates;
// request a rebuild when an atom moved more than skin/2 since the last build.
__global__ void md_drift_kernel(int N, double *x, double *v, const double *F, float4 *pos4, const double *x_ref,
                                const double *origin, const double *inv_mass_kappa, double dt, double half_skin2,
                                BuildStatus *st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) st->md_steps += 1;
  if (i >= N) return;
  float4 p = pos4[i];
  const double s = 0.5 * dt * inv_mass_kappa[type_of(p)];
  double r[3], d2 = 0.0;
  for (int b = 0; b < 3; ++b) {
    const size_t k = 3 * (size_t)i + b;
    const double vb = v[k] + s * F[k];
    v[k] = vb;
    r[b] = x[k] + dt * vb;
    x[k] = r[b];
    const double dd = r[b] - x_ref[k];
    d2 += dd * dd;
  }
  p.x = (float)(r[0] - origin[3 * (size_t)i]);
  p.y = (float)(r[1] - origin[3 * (size_t)i + 1]);
  p.z = (float)(r[2] - origin[3 * (size_t)i + 2]);
  pos4[i] = p;
  if (d2 > half_skin2) st->rebuild = 1;
}

// Deterministic totals: E = sum U_i, W = sum W_i, kinetic energy; optional thermo row.
// One block; every thread sums a fixed strided subset, then a fixed tree.
__global__ void finalize_kernel(int nb_atom, const double *partial_atom, int nb_gather, const double *partial_gather,
                                double *energy_total, double *virial_total, double *thermo_stage,
                                int *thermo_ctl /* [0] step-in-call, [1] rows written, [2] every */, int N,
                                double volume) {
  __shared__ double red[256][kReduceSlots];
  double acc[kReduceSlots];
  for (int s = 0; s < kReduceSlots; ++s) acc[s] = 0.0;
  for (int b = threadIdx.x; b < nb_atom; b += blockDim.x) acc[0] += partial_atom[b];
  for (int b = threadIdx.x; b < nb_gather; b += blockDim.x)
    for (int s = 1; s < 11; ++s) acc[s] += partial_gather[(size_t)b * kReduceSlots + s];
  for (int s = 0; s < kReduceSlots; ++s) red[threadIdx.x][s] = acc[s];
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int s = 0; s < kReduceSlots; ++s) red[threadIdx.x][s] += red[threadIdx.x + off][s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (energy_total) *energy_total = red[0][0];
    if (virial_total)
      for (int c = 0; c < 9; ++c) virial_total[c] = red[0][2 + c];
    if (thermo_ctl) {
      const int step = ++thermo_ctl[0];
      if (step % thermo_ctl[2] == 0) {
        const int row = thermo_ctl[1]++;
        const double kb = 8.617333262e-5;
        const double ke = red[0][1];
        const double tr = red[0][2] + red[0][3] + red[0][4];
        double *o = thermo_stage + 4 * (size_t)row;
        o[0] = red[0][0];
        o[1] = ke;
        o[2] = N > 1 ? 2.0 * ke / ((3.0 * N - 3.0) * kb) : 0.0;
        o[3] = (2.0 * ke + tr) / (3.0 * volume) * 160.21766208;  // eV/A^3 -> GPa
      }
    }
  }
}

// Positions wrapped into the cell (fractional coordinates in [0, 1)).
__global__ void wrap_positions_kernel(int N, const double *x, const Grid g, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double r[3] = {x[3 * (size_t)i], x[3 * (size_t)i + 1], x[3 * (size_t)i + 2]};
  double s[3];
  for (int b = 0; b < 3; ++b) {
    s[b] = r[0] * g.Hinv[0][b] + r[1] * g.Hinv[1][b] + r[2] * g.Hinv[2][b];
    s[b] -= floor(s[b]);
  }
  for (int b = 0; b < 3; ++b) out[3 * (size_t)i + b] = s[0] * g.H[0][b] + s[1] * g.H[1][b] + s[2] * g.H[2][b];
}

// ------------------------------------------------------------------ host launchers
void launch_wrap(int N, const double *x, const Grid &g, double *out, cudaStream_t s) {
  wrap_positions_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, x, g, out);
}

void launch_rebuild(int N, int T, const Grid &g, const float4 *dtab, float rlR2, float rlA2, float rcR2, float rcA2,
                    int cap_r, int cap_a,
                    int count_only, double *x, double *x_ref, double *origin, const int *types, float4 *pos4,
                    int *cell_of, int *cell_count, int *cell_cursor, int *cell_start, int *cell_atoms,
                    unsigned *nl_r, int *nn_r, unsigned *nl_a, int *nn_a, int *rev_a, BuildStatus *st,
                    cudaStream_t s) {
  const int tb = 256;
  const int nb = (N + tb - 1) / tb;
  const int cb = (g.ncell + tb - 1) / tb;
  zero_cells_kernel<<<cb < 1024 ? cb : 1024, tb, 0, s>>>(g.ncell, cell_count, cell_cursor, st);
  bin_atoms_kernel<<<nb, tb, 0, s>>>(N, T, x, x_ref, origin, types, pos4, cell_of, cell_count, g, st);
  scan_cells_kernel<<<1, 1024, 0, s>>>(g.ncell, cell_count, cell_start, st);
  scatter_atoms_kernel<<<nb, tb, 0, s>>>(N, cell_of, cell_start, cell_cursor, cell_atoms, st);
  sort_cells_kernel<<<cb, tb, 0, s>>>(g.ncell, cell_start, cell_atoms, st);
  build_lists_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, pos4, cell_of, cell_start, cell_atoms, g, dtab, rlR2, rlA2, rcR2,
                                                     rcA2, T, cap_r, cap_a, count_only, nl_r, nn_r, nl_a, nn_a, st);
  if (!count_only) build_rev_kernel<<<nb, tb, 0, s>>>(N, nl_a, nn_a, g, rev_a, st);
  finish_build_kernel<<<1, 1, 0, s>>>(st);
}

void launch_drift(int N, double *x, double *v, const double *F, float4 *pos4, const double *x_ref,
                  const double *origin, const double *inv_mass_kappa, double dt, double half_skin2, BuildStatus *st,
                  cudaStream_t s) {
  md_drift_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, x, v, F, pos4, x_ref, origin, inv_mass_kappa, dt, half_skin2, st);
}

void launch_finalize(int nb_atom, const double *partial_atom, int nb_gather, const double *partial_gather,
                     double *energy_total, double *virial_total, double *thermo_stage, int *thermo_ctl, int N,
                     double volume, cudaStream_t s) {
  finalize_kernel<<<1, 256, 0, s>>>(nb_atom, partial_atom, nb_gather, partial_gather, energy_total, virial_total,
                                    thermo_stage, thermo_ctl, N, volume);
}

}  // namespace nep
