// Neighbour-list construction, atom reordering, velocity-Verlet drift and reductions.
//
// The paper takes its neighbour lists as given (Appendix B lists NN_i^R, NN_i^A, NL_im^R,
// NL_im^A); here they are built on the GPU from a cell list at every rebuild:
//   bin_atoms      validate, wrap positions into the cell (FP64), cell index, cell counts;
//   scan_cells     exclusive prefix sum of the counts (one block, deterministic);
//   scatter/sort   atoms into their cells, each cell ordered by atom index (deterministic);
//   reorder        move every per-atom array into cell order (the internal order), so a
//                  warp's atoms are spatial neighbours and their neighbour data is shared in
//                  L1; perm keeps the caller's index of each internal atom;
//   commit         cell-local FP32 coordinates, cell origins, reference positions;
//   build_lists    per atom: scan the (2R+1)^3 neighbouring cells (all periodic images when
//                  the cell is thin), keep pairs within r_c + skin, group the radial list by
//                  neighbour type and put the pairs inside r_c before the skin pairs (which
//                  keeps warps convergent in the pair loops); two passes, count then write;
//   build_rev      for every angular pair (i, j, image), the slot of (j, i, -image) in the list
//                  of j, so forces are gathered without atomics (Algorithm 4's "index
//                  manipulations").
// Every builder returns early unless a rebuild is pending, so the whole sequence sits in the
// captured MD step graph and only works when an atom moved more than skin/2. In the serving
// engine's batch a build that was not forced covers only the structures whose atoms moved that
// far (per-structure flags); the others keep their cells, atom order, lists and x_ref.
#include <cuda_bf16.h>

#include "nep_internal.cuh"

namespace nep {

// Grid of the structure that atom i belongs to.
__device__ __forceinline__ const Grid &grid_of(const Batch &B, const Grid &g, int i) {
  return B.grids ? B.grids[B.sid[i]] : g;
}

__device__ __forceinline__ bool rebuild_pending(const BuildStatus *st) {
  return *(volatile const int *)&st->rebuild != 0;
}

// Atom (or internal position) i belongs to a structure that this build leaves as it is: a
// build requested by the serving engine's drift kernel, not forced, and i's structure not
// flagged. Such atoms keep their cell, their place in the order, their lists and x_ref.
__device__ __forceinline__ bool kept_by_build(const Batch &B, const BuildStatus *st, int i) {
  return B.sflag && !*(volatile const int *)&st->full && B.sflag[B.sid[i]] == 0;
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

__global__ void bin_atoms_kernel(int N, int T, AtomState a, int *count, const Grid g0, const Batch B,
                                 BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (kept_by_build(B, st, i)) {  // counted in its old cell: its structure's order stays
    atomicAdd(count + a.cell_of[i], 1);
    return;
  }
  const Grid &g = grid_of(B, g0, i);
  double *x = a.x + 3 * (size_t)i;
  double r[3] = {x[0], x[1], x[2]};
  const int ti = a.types[i];
  if (ti < 0 || ti >= T) {
    atomicOr(&st->bad_input, 1);
    a.types[i] = 0;
  }
  bool inside = true;
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2])) {
    atomicOr(&st->bad_input, 2);
    r[0] = r[1] = r[2] = 0.0;
    inside = false;  // overwrite the position
  }
  double s[3];
  int c[3];
  for (int b = 0; b < 3; ++b) {
    s[b] = r[0] * g.Hinv[0][b] + r[1] * g.Hinv[1][b] + r[2] * g.Hinv[2][b];
    const double f = floor(s[b]);
    inside = inside && f == 0.0;
    s[b] -= f;
    const int cb = (int)(s[b] * g.nc[b]);
    c[b] = cb < 0 ? 0 : (cb >= g.nc[b] ? g.nc[b] - 1 : cb);
  }
  // only atoms outside the cell are moved (a position is not re-rounded by every build)
  if (!inside)
    for (int b = 0; b < 3; ++b) x[b] = s[0] * g.H[0][b] + s[1] * g.H[1][b] + s[2] * g.H[2][b];
  const int id = g.cell_off + (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  a.cell_of[i] = id;
  atomicAdd(count + id, 1);
}

// Exclusive prefix sum of the cell counts by one block of 1024 threads, in tiles of 4096
// cells: every thread takes 4 consecutive counts (one 16-byte load), the block scans the
// thread totals (warp shuffles, then the warp totals) and carries the tile total on.
__global__ void scan_cells_kernel(int ncell, const int *count, int *start, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int carry = 0;
  for (int base = 0; base < ncell; base += 4 * 1024) {
    const int c0 = base + 4 * threadIdx.x;
    int v[4];
    if (c0 + 3 < ncell) {
      const int4 q = *reinterpret_cast<const int4 *>(count + c0);
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = c0 + k < ncell ? count[c0 + k] : 0;
    }
    const int tot = (v[0] + v[1]) + (v[2] + v[3]);
    int x = tot;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int run = carry + (wid > 0 ? wsum[wid - 1] : 0) + (x - tot);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (c0 + k < ncell) start[c0 + k] = run;
      run += v[k];
    }
    carry += wsum[31];
    __syncthreads();  // wsum is rewritten by the next tile
  }
  if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void scatter_atoms_kernel(int N, const int *cell_of, const int *start, int *cursor, int *cell_atoms,
                                     const Batch B, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || kept_by_build(B, st, i)) return;
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

// Internal atom p takes the data of atom cell_atoms[p] (into the scratch arrays).
__global__ void reorder_gather_kernel(int N, const int *cell_atoms, AtomState a, const Batch B,
                                      const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N || kept_by_build(B, st, p)) return;
  const int o = cell_atoms[p];
  for (int b = 0; b < 3; ++b) {
    a.x2[3 * (size_t)p + b] = a.x[3 * (size_t)o + b];
    a.v2[3 * (size_t)p + b] = a.v[3 * (size_t)o + b];
    a.F2[3 * (size_t)p + b] = a.F[3 * (size_t)o + b];
  }
  a.types2[p] = a.types[o];
  a.perm2[p] = a.perm[o];
  a.cell2[p] = a.cell_of[o];
}

// Copy the reordered data back and derive the cell-local coordinates.
__global__ void reorder_commit_kernel(int N, AtomState a, const Grid g0, const Batch B, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N || kept_by_build(B, st, p)) return;
  // cells are numbered structure by structure, so atom p stays inside its structure's range
  const Grid &g = grid_of(B, g0, p);
  const int gid = a.cell2[p];
  const int id = gid - g.cell_off;
  const int c0 = id / (g.nc[1] * g.nc[2]), c1 = (id / g.nc[2]) % g.nc[1], c2 = id % g.nc[2];
  double r[3], o[3];
  for (int b = 0; b < 3; ++b) {
    r[b] = a.x2[3 * (size_t)p + b];
    o[b] = c0 * g.Hc[0][b] + c1 * g.Hc[1][b] + c2 * g.Hc[2][b];
    a.x[3 * (size_t)p + b] = r[b];
    a.x_ref[3 * (size_t)p + b] = r[b];
    a.origin[3 * (size_t)p + b] = o[b];
    a.v[3 * (size_t)p + b] = a.v2[3 * (size_t)p + b];
    a.F[3 * (size_t)p + b] = a.F2[3 * (size_t)p + b];
  }
  const int t = a.types2[p];
  a.types[p] = t;
  a.perm[p] = a.perm2[p];
  a.cell_of[p] = gid;
  const int sidp = B.grids ? B.sid[p] : 0;
  a.pos4[p] = make_float4((float)(r[0] - o[0]), (float)(r[1] - o[1]), (float)(r[2] - o[2]),
                          __int_as_float(t | (sidp << 8)));
  a.posA[p] = make_float4((float)r[0], (float)r[1], (float)r[2], __int_as_float(t | (sidp << 8)));
}

// floor(x / n) and the remainder, for n >= 1 and x > -n * 8
__device__ __forceinline__ int floor_div(int x, int n) { return (x + 8 * n) / n - 8; }

// Visit every neighbour candidate (j, image) of atom i: f(j, entry, r2, type_j). Atoms are in
// cell order, so the atoms of cell c are j in [start[c], start[c+1]). For each (x, y) column of
// neighbouring cells the z cells are walked as runs that share one periodic image, so the
// shift S is formed once per run and the distance comes from the FP32 positions in the cell
// frame: d = (r_j - r_i) + S, exactly antisymmetric like pair_vector. The image code of an
// entry is the cell offset (ox, oy, oz), as the force kernels' shift tables expect.
//
// Cells that cannot hold a pair are skipped: along axis a, atom i sits at the fraction u_a of
// its cell's width, so every point of the cell at offset o >= 1 lies (o - u_a) cell
// thicknesses away across the lattice planes, and of the cell at o <= -1, (u_a - o - 1); a
// cell is visited only if that gap stays below reach_a = (r_c^R + skin + margin) / thickness.
// The skipped candidates would all fail the distance test, so the lists (and their order)
// are those of the full (2R+1)^3 scan. pl: atom i's cell-local coordinates (pos4).
template <class F>
__device__ __forceinline__ void for_candidates(int i, const float4 &pi, const float4 &pl, int gid, const Grid &g,
                                               const int *start, const float4 *posA, F &&f) {
  const int id = gid - g.cell_off;
  const int cx = id / (g.nc[1] * g.nc[2]);
  const int cy = (id / g.nc[2]) % g.nc[1];
  const int cz = id % g.nc[2];
  float Hf[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Hf[a][b] = (float)g.H[a][b];
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float s = pl.x * (float)g.Hinv[0][a] + pl.y * (float)g.Hinv[1][a] + pl.z * (float)g.Hinv[2][a];
    const float u = fminf(fmaxf(s * (float)g.nc[a], 0.f), 1.f);
    hi[a] = min(g.R[a], (int)ceilf(u + g.reach[a]) - 1);
    lo[a] = max(-g.R[a], 1 - (int)ceilf(1.f - u + g.reach[a]));
  }
  for (int ox = lo[0]; ox <= hi[0]; ++ox) {
    const int kx = floor_div(cx + ox, g.nc[0]);
    const int xm = cx + ox - kx * g.nc[0];
    for (int oy = lo[1]; oy <= hi[1]; ++oy) {
      const int ky = floor_div(cy + oy, g.nc[1]);
      const int ym = cy + oy - ky * g.nc[1];
      const int col = g.cell_off + (xm * g.nc[1] + ym) * g.nc[2];
      const float sx = __fadd_rn(__fmul_rn((float)kx, Hf[0][0]), __fmul_rn((float)ky, Hf[1][0]));
      const float sy = __fadd_rn(__fmul_rn((float)kx, Hf[0][1]), __fmul_rn((float)ky, Hf[1][1]));
      const float sz = __fadd_rn(__fmul_rn((float)kx, Hf[0][2]), __fmul_rn((float)ky, Hf[1][2]));
      const unsigned code_xy = (unsigned)(ox + g.R[0]) | ((unsigned)(oy + g.R[1]) << g.obits);
      int z = cz + lo[2];
      while (z <= cz + hi[2]) {
        const int kz = floor_div(z, g.nc[2]);
        const int zm = z - kz * g.nc[2];
        const int run = min(cz + hi[2] - z, g.nc[2] - 1 - zm) + 1;  // cells of this image
        const float4 S = make_float4(__fadd_rn(sx, __fmul_rn((float)kz, Hf[2][0])),
                                     __fadd_rn(sy, __fmul_rn((float)kz, Hf[2][1])),
                                     __fadd_rn(sz, __fmul_rn((float)kz, Hf[2][2])), 0.f);
        for (int c = 0; c < run; ++c) {
          const int oz = z + c - cz;
          const unsigned code = code_xy | ((unsigned)(oz + g.R[2]) << (2 * g.obits));
          const bool self_image = (ox == 0 && oy == 0 && oz == 0);
          const int cell = col + zm + c;
          const int pe = start[cell + 1];
          for (int j = start[cell]; j < pe; ++j) {
            if (self_image && j == i) continue;
            const float4 pj = posA[j];
            f(j, (unsigned)j | (code << g.jbits), norm2(pair_vector(pi, pj, S)), type_of(pj));
          }
        }
        z += run;
      }
    }
  }
}

// Two passes over the candidates: count, then write. The radial list is grouped by
// neighbour type; inside every group (and in the angular list) the pairs already inside
// r_c come before the skin pairs, so the warps of the pair loops stay convergent.
// count_only: record only the length statistics (used to size the lists). TT: the number of
// atom types (compile time, so the per-type counters of a candidate cost TT compares).
template <int TT>
__global__ void build_lists_kernel(int N, const float4 *posA, const float4 *pos4, const int *cell_of, const int *start,
                                   const Grid g0, const Batch B, float rlR2, float rlA2, float rcR2, float rcA2,
                                   ListBufs L, int count_only, BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  // lanes past the last atom (and atoms of structures this build keeps) stay until the
  // warp-level statistics below
  const bool active = i0 < N && !kept_by_build(B, st, i0);
  const int i = active ? i0 : 0;  // a valid index for the idle lanes (N >= 1)
  const Grid &g = grid_of(B, g0, i);
  const float4 pi = posA[i];
  const float4 pl = pos4[i];
  const int id = cell_of[i];
  // per-type counters stay in registers: every update is unrolled over the types
  int cr0[TT], cr1[TT];
#pragma unroll
  for (int t = 0; t < TT; ++t) cr0[t] = cr1[t] = 0;
  int ca0 = 0, ca1 = 0;
  // with a staging area the accepted candidates are kept in visiting order together with
  // their group (type, inside r_c or skin, angular or not), so the lists are written from
  // them instead of a second candidate scan
  const bool staged = !count_only && L.stage_e;
  int n_seen = 0;
  if (active && staged) {
    // the scan only stages the accepted candidates (angular pairs are a subset of the radial
    // ones, r_c^A <= r_c^R); their groups are counted afterwards from the staged bytes
    unsigned *se = L.stage_e + i;
    unsigned char *sg = L.stage_g + i;
    for_candidates(i, pi, pl, id, g, start, posA, [&](int, unsigned ent, float r2, int tj) {
      if (r2 < rlR2) {
        if (n_seen < L.cap_r) {
          const int ang = r2 < rlA2 ? (r2 < rcA2 ? 1 : 2) : 0;
          *se = ent;
          *sg = (unsigned char)(tj | (r2 < rcR2 ? 0 : 8) | (ang << 4));
          se += N;
          sg += N;
        }
        ++n_seen;
      }
    });
    const int ns = n_seen < L.cap_r ? n_seen : L.cap_r;
    for (int m = 0; m < ns; ++m) {
      const unsigned gb = L.stage_g[(size_t)m * N + i];
      const int tj = (int)(gb & 7u);
      const bool core = (gb & 8u) == 0;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        cr0[t] += (tj == t && core) ? 1 : 0;
        cr1[t] += (tj == t && !core) ? 1 : 0;
      }
      const unsigned ang = gb >> 4;
      ca0 += ang == 1u ? 1 : 0;
      ca1 += ang == 2u ? 1 : 0;
    }
    // past the staging capacity the groups are unknown: the build overflows and is redone
    // with lists sized from these counts (the unstaged pairs counted as skin pairs of type 0,
    // and as angular ones, an upper bound)
    cr1[0] += n_seen - ns;
    ca1 += n_seen - ns;
  } else if (active) {
    for_candidates(i, pi, pl, id, g, start, posA, [&](int, unsigned ent, float r2, int tj) {
      if (r2 < rlR2) {
        const bool core = r2 < rcR2;
#pragma unroll
        for (int t = 0; t < TT; ++t) {
          cr0[t] += (tj == t && core) ? 1 : 0;
          cr1[t] += (tj == t && !core) ? 1 : 0;
        }
        ++n_seen;
      }
      if (r2 < rlA2) {
        if (r2 < rcA2) ++ca0;
        else ++ca1;
      }
    });
  }
  int nr = 0, inr = 0;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    nr += cr0[t] + cr1[t];
    inr += cr0[t];
  }
  const int nA = ca0 + ca1;
  // list statistics: reduced over the warp first, one atomic per warp and counter (every
  // thread updating the same few words serialises in the L2 atomic unit)
  {
    int mr = nr, ma = nA;
    unsigned long long sr = nr, sa = nA, ir = inr, ia = ca0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
      ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      ir += __shfl_xor_sync(0xffffffffu, ir, o);
      ia += __shfl_xor_sync(0xffffffffu, ia, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&st->max_r, mr);
      atomicMax(&st->max_a, ma);
      atomicAdd(&st->sum_r, sr);
      atomicAdd(&st->sum_a, sa);
      atomicAdd(&st->in_r, ir);
      atomicAdd(&st->in_a, ia);
    }
  }
  if (count_only || !active) return;
  if (nr > L.cap_r || nA > L.cap_a) {  // leave the lists empty; the host grows them and rebuilds
    atomicOr(&st->overflow, 1);
    for (int t = 0; t < TT; ++t) L.nn_r[t * N + i] = 0;
    L.nn_a[i] = 0;
    return;
  }
  int cur0[TT], cur1[TT];
  int off = 0;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    cur0[t] = off;
    cur1[t] = off + cr0[t];
    off += cr0[t] + cr1[t];
    L.nn_r[t * N + i] = cr0[t] + cr1[t];
  }
  int ka0 = 0, ka1 = ca0;
  if (staged) {
    for (int m = 0; m < nr; ++m) {
      const unsigned ent = L.stage_e[(size_t)m * N + i];
      const unsigned gb = L.stage_g[(size_t)m * N + i];
      const int tj = (int)(gb & 7u);
      const bool core = (gb & 8u) == 0;
      int slot = 0;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        if (tj == t) {
          slot = core ? cur0[t] : cur1[t];
          cur0[t] += core ? 1 : 0;
          cur1[t] += core ? 0 : 1;
        }
      }
      L.nl_r[(size_t)slot * N + i] = ent;
      const unsigned ang = gb >> 4;
      if (ang) L.nl_a[(size_t)(ang == 1u ? ka0++ : ka1++) * N + i] = ent;
    }
    L.nn_a[i] = nA;
    return;
  }
  for_candidates(i, pi, pl, id, g, start, posA, [&](int, unsigned ent, float r2, int tj) {
    if (r2 < rlR2) {
      const bool core = r2 < rcR2;
      int slot = 0;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        if (tj == t) {
          slot = core ? cur0[t] : cur1[t];
          cur0[t] += core ? 1 : 0;
          cur1[t] += core ? 0 : 1;
        }
      }
      L.nl_r[(size_t)slot * N + i] = ent;
    }
    if (r2 < rlA2) L.nl_a[(size_t)(r2 < rcA2 ? ka0++ : ka1++) * N + i] = ent;
  });
  L.nn_a[i] = nA;
}

__global__ void build_rev_kernel(int N, const ListBufs L, const Grid g0, const Batch B, BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || kept_by_build(B, st, i)) return;
  const Grid &g = grid_of(B, g0, i);
  const unsigned om = (1u << g.obits) - 1u;
  const int na = L.nn_a[i];
  for (int m = 0; m < na; ++m) {
    const size_t slot = (size_t)m * N + i;
    const unsigned e = L.nl_a[slot];
    const int j = e & g.jmask;
    const unsigned code = e >> g.jbits;
    const unsigned cx = code & om, cy = (code >> g.obits) & om, cz = (code >> (2 * g.obits)) & om;
    const unsigned rc = (2u * g.R[0] - cx) | ((2u * g.R[1] - cy) << g.obits) | ((2u * g.R[2] - cz) << (2 * g.obits));
    const unsigned target = (unsigned)i | (rc << g.jbits);
    const int nj = L.nn_a[j];
    int found = -1;
    for (int q = 0; q < nj; ++q)
      if (L.nl_a[(size_t)q * N + j] == target) {
        found = q;
        break;
      }
    if (found < 0) {
      atomicAdd(&st->rev_missing, 1);
      L.rev_a[slot] = (int)slot;  // a finite entry; the status reports the error
    } else {
      L.rev_a[slot] = (int)((size_t)found * N + j);
    }
  }
}

__global__ void finish_build_kernel(BuildStatus *st) {
  if (st->rebuild) {
    st->rebuild = 0;
    st->full = 0;
    st->n_rebuilds += 1;
  }
}

// The per-structure build requests are served: clear them (before finish_build_kernel).
__global__ void clear_sflags_kernel(int n_struct, int *sflag, const BuildStatus *st) {
  if (!rebuild_pending(st)) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_struct; s += gridDim.x * blockDim.x) sflag[s] = 0;
}

// Sets the condition of the graph's rebuild node from the drift kernel's request.
__global__ void rebuild_condition_kernel(cudaGraphConditionalHandle hc, const BuildStatus *st) {
  cudaGraphSetConditional(hc, *(volatile const int *)&st->rebuild != 0 ? 1u : 0u);
}

__global__ void iota_kernel(int N, int *perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) perm[i] = i;
}

// Velocity Verlet, first half: v += dt/2 F/m; x += dt v; refresh cell-local coordinates;
// request a rebuild when an atom moved more than skin/2 since the last build.
// With a FIRE state, its time step is used and a converged relaxation stays where it is.
__global__ void md_drift_kernel(int N, AtomState a, const double *inv_mass_kappa, double dt, double half_skin2,
                                BuildStatus *st, const FireState *fire) {
  if (fire) {
    if (fire->converged) return;
    dt = fire->dt;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) st->md_steps += 1;
  if (i >= N) return;
  float4 p = a.pos4[i];
  const double s = 0.5 * dt * inv_mass_kappa[type_of(p)];
  double r[3], d2 = 0.0;
  for (int b = 0; b < 3; ++b) {
    const size_t k = 3 * (size_t)i + b;
    const double vb = a.v[k] + s * a.F[k];
    a.v[k] = vb;
    r[b] = a.x[k] + dt * vb;
    a.x[k] = r[b];
    const double dd = r[b] - a.x_ref[k];
    d2 += dd * dd;
  }
  p.x = (float)(r[0] - a.origin[3 * (size_t)i]);
  p.y = (float)(r[1] - a.origin[3 * (size_t)i + 1]);
  p.z = (float)(r[2] - a.origin[3 * (size_t)i + 2]);
  a.pos4[i] = p;
  if (d2 > half_skin2) st->rebuild = 1;
}

// Caller-order copies of the MD state: positions wrapped into the cell, velocities, forces.
__global__ void export_state_kernel(int N, const AtomState a, const Grid g0, const Batch B, double *pos, double *vel,
                                    double *force) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Grid &g = grid_of(B, g0, i);
  const size_t u = 3 * (size_t)a.perm[i];
  if (pos) {
    const double r[3] = {a.x[3 * (size_t)i], a.x[3 * (size_t)i + 1], a.x[3 * (size_t)i + 2]};
    double s[3];
    for (int b = 0; b < 3; ++b) {
      s[b] = r[0] * g.Hinv[0][b] + r[1] * g.Hinv[1][b] + r[2] * g.Hinv[2][b];
      s[b] -= floor(s[b]);
    }
    for (int b = 0; b < 3; ++b) pos[u + b] = s[0] * g.H[0][b] + s[1] * g.H[1][b] + s[2] * g.H[2][b];
  }
  for (int b = 0; b < 3; ++b) {
    if (vel) vel[u + b] = a.v[3 * (size_t)i + b];
    if (force) force[u + b] = a.F[3 * (size_t)i + b];
  }
}

// Deterministic totals: E = sum U_i, W = sum W_i, kinetic energy, heat current J = sum J_i;
// optional thermo row. One block; every thread sums a fixed strided subset, then a fixed
// tree. In MD mode (thermo_ctl set) steps without a thermo row only advance the step
// counter. A thermo row holds E_pot, E_kin, T, P, J_x, J_y, J_z and the thermostat factor;
// with a thermostat (ts) the kinetic energy is that after the step's velocity rescaling.
constexpr int kThermoCols = 8;

__global__ void finalize_kernel(int nb_atom, const double *partial_atom, int nb_gather, const double *partial_gather,
                                double *energy_total, double *virial_total, double *heat_total,
                                double *thermo_stage, int *thermo_ctl /* [0] step-in-call, [1] rows written, [2] every */,
                                int N, double volume, const ThermoState *ts) {
  __shared__ double red[256][kReduceSlots];
  __shared__ int emit;
  if (threadIdx.x == 0) {
    emit = 1;
    if (thermo_ctl) {
      const int step = ++thermo_ctl[0];
      emit = (step % thermo_ctl[2] == 0);
    }
  }
  __syncthreads();
  if (!emit) return;
  double acc[kReduceSlots];
  for (int s = 0; s < kReduceSlots; ++s) acc[s] = 0.0;
  for (int b = threadIdx.x; b < nb_atom; b += blockDim.x) acc[0] += partial_atom[b];
  for (int b = threadIdx.x; b < nb_gather; b += blockDim.x)
    for (int s = 1; s < kReduceSlots; ++s) acc[s] += partial_gather[(size_t)b * kReduceSlots + s];
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
    if (heat_total)
      for (int c = 0; c < 3; ++c) heat_total[c] = red[0][12 + c];
    if (thermo_ctl) {
      const int row = thermo_ctl[1]++;
      const double kb = 8.617333262e-5;
      const double alpha = ts ? ts->alpha : 1.0;
      const double ke = red[0][1] * alpha * alpha;
      const double tr = red[0][2] + red[0][3] + red[0][4];
      double *o = thermo_stage + kThermoCols * (size_t)row;
      o[0] = red[0][0];
      o[1] = ke;
      o[2] = N > 1 ? 2.0 * ke / ((3.0 * N - 3.0) * kb) : 0.0;
      o[3] = (2.0 * ke + tr) / (3.0 * volume) * 160.21766208;  // eV/A^3 -> GPa
      // J with the rescaled velocities: J is linear in v
      for (int c = 0; c < 3; ++c) o[4 + c] = red[0][12 + c] * alpha;
      o[7] = alpha;
    }
  }
}

// Bussi-Donadio-Parrinello rescaling after a velocity-Verlet step: K from the gather
// kernel's block sums (fixed order), then with c = exp(-dt/tau), Kbar = N_f k_B T0 / 2 and
// this step's R1, S: alpha^2 = c + (1 - c)(S + R1^2) Kbar / (N_f K)
//                              + 2 R1 sqrt(c (1 - c) Kbar / (N_f K)),
// alpha taking the sign of R1 + sqrt(c N_f K / ((1 - c) Kbar)); then v <- alpha v.
__global__ void thermostat_factor_kernel(int nb_gather, const double *partial_gather, ThermoState *ts) {
  __shared__ double red[256];
  double k = 0.0;
  for (int b = threadIdx.x; b < nb_gather; b += blockDim.x) k += partial_gather[(size_t)b * kReduceSlots + 1];
  red[threadIdx.x] = k;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double K = red[0], c = ts->c, kbar = ts->kbar, nf = ts->nf;
    const double R1 = ts->rand[2 * ts->step], S = ts->rand[2 * ts->step + 1];
    double alpha = 1.0;
    if (K > 0.0) {
      const double q = kbar / (nf * K);
      const double a2 = c + (1.0 - c) * (S + R1 * R1) * q + 2.0 * R1 * sqrt(c * (1.0 - c) * q);
      alpha = sqrt(fmax(a2, 0.0));
      if (c < 1.0 && R1 + sqrt(c / ((1.0 - c) * q)) < 0.0) alpha = -alpha;
    }
    ts->alpha = alpha;
    ts->step += 1;
  }
}

__global__ void scale_velocities_kernel(int N, double *v, const ThermoState *ts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = ts->alpha;
  for (int b = 0; b < 3; ++b) v[3 * (size_t)i + b] *= a;
}

void launch_thermostat(int N, const AtomState &a, int nb_gather, const double *partial_gather, ThermoState *ts,
                       cudaStream_t s) {
  thermostat_factor_kernel<<<1, 256, 0, s>>>(nb_gather, partial_gather, ts);
  scale_velocities_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, a.v, ts);
}

// ------------------------------------------------------------------ batches
// Structure s owns the atoms [offsets[s], offsets[s+1]) in the caller's order, and (the
// cells being numbered structure by structure) the same range in the internal order.
__global__ void struct_ids_kernel(int n_struct, const int *offsets, int *sid) {
  const int s = blockIdx.x;
  if (s >= n_struct) return;
  for (int i = offsets[s] + threadIdx.x; i < offsets[s + 1]; i += blockDim.x) sid[i] = s;
}

// Shift vector of every image code of every structure (zero for codes outside the range).
__global__ void shift_tables_kernel(int n_struct, const Grid *grids, int ncode, int obits, float4 *dtab) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)n_struct * ncode) return;
  const int s = (int)(v / ncode), code = (int)(v % ncode);
  const Grid &g = grids[s];
  const int om = (1 << obits) - 1;
  const int o[3] = {(code & om) - g.R[0], ((code >> obits) & om) - g.R[1], ((code >> (2 * obits)) & om) - g.R[2]};
  float4 D = make_float4(0.f, 0.f, 0.f, 0.f);
  if (abs(o[0]) <= g.R[0] && abs(o[1]) <= g.R[1] && abs(o[2]) <= g.R[2]) {
    double d[3];
    for (int b = 0; b < 3; ++b)
      d[b] = __dadd_rn(__dadd_rn(__dmul_rn(o[0], g.Hc[0][b]), __dmul_rn(o[1], g.Hc[1][b])), __dmul_rn(o[2], g.Hc[2][b]));
    D = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
  }
  dtab[g.dtab_off + code] = D;
}

// Per-structure sums E_s = sum U_i and W_s = sum W_i (FP64, fixed order). A structure of at
// most kWideSum atoms takes one warp (WIDE = false); a larger one one block of kSumThreads
// threads (WIDE = true), so its FP64 additions run on eight warps. Every thread adds a fixed
// stride of the structure's atoms into four partial sums by round (round mod 4: independent
// chains), combined in a fixed order, then a fixed shuffle tree (and, wide, the warp totals in
// warp order): the result depends only on the structure's atom range.
constexpr int kWideSum = 2048;
constexpr int kSumThreads = 256;
template <bool WIDE>
__global__ void struct_sums_kernel(int n_struct, int members, const int *offsets, int N, const double *e_atom,
                                   const double *w_atom, double *e_struct, double *w_struct) {
  const int lane = threadIdx.x & 31;
  const long long unit = WIDE ? (long long)blockIdx.x : ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (unit >= (long long)n_struct * members) return;  // uniform over the warp (block, WIDE)
  const int m = (int)(unit / n_struct), s = (int)(unit % n_struct);
  const int a0 = offsets[s], a1 = offsets[s + 1];
  if ((a1 - a0 > kWideSum) != WIDE) return;  // the other form takes this structure
  const size_t base = (size_t)m * N;
  const int t = WIDE ? (int)threadIdx.x : lane, nt = WIDE ? kSumThreads : 32;
  double acc[4][10];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[r][c] = 0.0;
  auto add = [&](double *a, size_t k) {
    if (e_atom) a[0] += e_atom[k];
    if (w_atom)
#pragma unroll
      for (int c = 0; c < 9; ++c) a[1 + c] += w_atom[9 * k + c];
  };
  int i = a0 + t;
  for (; i + 3 * nt < a1; i += 4 * nt) {  // four rounds at a time
#pragma unroll
    for (int r = 0; r < 4; ++r) add(acc[r], base + i + (size_t)nt * r);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)  // at most three rounds left
    if (i < a1) {
      add(acc[r], base + i);
      i += nt;
    }
  double tot[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    tot[c] = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot[c] += __shfl_down_sync(0xffffffffu, tot[c], o);
  }
  const size_t o = (size_t)m * n_struct + s;
  if constexpr (WIDE) {
    __shared__ double red[kSumThreads / 32][10];
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < 10; ++c) red[threadIdx.x >> 5][c] = tot[c];
    __syncthreads();
    if (threadIdx.x < 10) {
      double v = 0.0;
      for (int w = 0; w < kSumThreads / 32; ++w) v += red[w][threadIdx.x];
      if (threadIdx.x == 0) {
        if (e_struct) e_struct[o] = v;
      } else if (w_struct) {
        w_struct[9 * o + threadIdx.x - 1] = v;
      }
    }
  } else if (lane == 0) {
    if (e_struct) e_struct[o] = tot[0];
    if (w_struct)
#pragma unroll
      for (int c = 0; c < 9; ++c) w_struct[9 * o + c] = tot[1 + c];
  }
}

// Marks a rebuild as pending and clears the per-build flags (the device form of the host
// reset before a forced rebuild, for captured graphs).
__global__ void arm_rebuild_kernel(BuildStatus *st) {
  st->overflow = 0;
  st->max_r = 0;
  st->max_a = 0;
  st->rev_missing = 0;
  st->bad_input = 0;
  st->tc_timeout = 0;
  st->rebuild = 1;
  st->full = 1;
}

// ------------------------------------------------------------------ population evaluation
// Candidate parameter vectors z [P][N_par], in the order c^R, c^A, w0, b0, w1, b1, become
// the FP32 arrays of the batched kernels (c^R, c^A and the network [w0 | b0 | w1 | b1]);
// reg[m] = (sum |z|, sum z^2) for the regularisation terms of Eq. loss. One block per member.
__global__ void unpack_population_kernel(const double *z, int n_par, int n_cr, int n_ca, float *cr, float *ca,
                                         float *ann, double *reg) {
  const int m = blockIdx.x;
  const int n_ann = n_par - n_cr - n_ca;
  const double *zm = z + (size_t)m * n_par;
  double s1 = 0.0, s2 = 0.0;
  for (int v = threadIdx.x; v < n_par; v += blockDim.x) {
    const double x = zm[v];
    s1 += fabs(x);
    s2 += x * x;
    if (v < n_cr) cr[(size_t)m * n_cr + v] = (float)x;
    else if (v < n_cr + n_ca) ca[(size_t)m * n_ca + (v - n_cr)] = (float)x;
    else ann[(size_t)m * n_ann + (v - n_cr - n_ca)] = (float)x;
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    reg[2 * m] = r1[0];
    reg[2 * m + 1] = r2[0];
  }
}

// BF16 operand tiles of every member's w0 (the layout of the single-model tiles): tile 1
// [NP1 x KP1] holds (mu, nu) -> w0[mu][nu], tile 2 [KP1 x NP1] holds (nu, mu) -> w0[mu][nu].
// The tiles must be zeroed before (padding).
__global__ void population_tiles_kernel(int n_pop, const float *ann, int n_ann, int H, int D, int KP1, int NP1,
                                        unsigned short *tiles) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)n_pop * H * D) return;
  const int m = (int)(v / ((long long)H * D));
  const int r = (int)(v % ((long long)H * D));
  const int mu = r / D, nu = r % D;
  const float x = ann[(size_t)m * n_ann + r];
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const unsigned short b = __bfloat16_as_ushort(bh);
  const unsigned short bl = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(bh)));
  const size_t tile = (size_t)NP1 * KP1;
  // per member: B1, B2, then the split form's B1_lo, B2_lo
  unsigned short *t1 = tiles + (size_t)m * 4 * tile, *t2 = t1 + tile;
  auto off = [](int row, int k, int kc) { return ((row / 8) * kc + k / 8) * 64 + (row % 8) * 8 + (k % 8); };
  t1[off(mu, nu, KP1 / 8)] = b;
  t2[off(nu, mu, NP1 / 8)] = b;
  t1[2 * tile + off(mu, nu, KP1 / 8)] = bl;
  t2[2 * tile + off(nu, mu, NP1 / 8)] = bl;
}

// Eq. loss for `members` candidates (one block each, fixed-order sums): RMSE of the energy
// per atom over the non-empty structures, RMSE of the force components (from the gather
// kernel's per-block sums), RMSE of the six virial components per atom (symmetric part of
// W_s / N_s; skipped without targets), and the l1 / l2 regularisation of z.
// loss[m] = (L, RMSE_E, RMSE_F, RMSE_W, sum|z| / N_par, sqrt(sum z^2 / N_par)).
__global__ void population_loss_kernel(int n_struct, const int *offsets, const double *e_struct,
                                       const double *w_struct, const double *e_tar, const double *w_tar,
                                       const double *partial_gather, int nb_gather, int N, const double *reg,
                                       int n_par, double le, double lf, double lv, double l1, double l2,
                                       double *loss) {
  const int m = blockIdx.x;
  double se = 0.0, sv = 0.0, sf = 0.0, cnt = 0.0;
  for (int s = threadIdx.x; s < n_struct; s += blockDim.x) {
    const int n = offsets[s + 1] - offsets[s];
    if (n <= 0) continue;
    cnt += 1.0;
    const double inv = 1.0 / n;
    const double de = e_struct[(size_t)m * n_struct + s] * inv - e_tar[s];
    se += de * de;
    if (w_struct && w_tar) {
      const double *w = w_struct + 9 * ((size_t)m * n_struct + s);
      const double sym[6] = {w[0], w[1], w[2], 0.5 * (w[3] + w[6]), 0.5 * (w[5] + w[8]), 0.5 * (w[4] + w[7])};
      for (int c = 0; c < 6; ++c) {
        const double dw = sym[c] * inv - w_tar[6 * (size_t)s + c];
        sv += dw * dw;
      }
    }
  }
  for (int b = threadIdx.x; b < nb_gather; b += blockDim.x)
    sf += partial_gather[((size_t)m * nb_gather + b) * kReduceSlots + 11];
  __shared__ double red[4][256];
  red[0][threadIdx.x] = se;
  red[1][threadIdx.x] = sv;
  red[2][threadIdx.x] = sf;
  red[3][threadIdx.x] = cnt;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ns = red[3][0];
    const double rmse_e = ns > 0 ? sqrt(red[0][0] / ns) : 0.0;
    const double rmse_w = (ns > 0 && w_struct && w_tar) ? sqrt(red[1][0] / (6.0 * ns)) : 0.0;
    const double rmse_f = N > 0 ? sqrt(red[2][0] / (3.0 * N)) : 0.0;
    const double r1 = reg[2 * m] / n_par, r2 = sqrt(reg[2 * m + 1] / n_par);
    double *o = loss + 6 * (size_t)m;
    o[0] = le * rmse_e + lf * rmse_f + lv * rmse_w + l1 * r1 + l2 * r2;
    o[1] = rmse_e;
    o[2] = rmse_f;
    o[3] = rmse_w;
    o[4] = r1;
    o[5] = r2;
  }
}

void launch_arm_rebuild(BuildStatus *st, cudaStream_t s) { arm_rebuild_kernel<<<1, 1, 0, s>>>(st); }

void launch_unpack_population(int n_pop, const double *z, int n_par, int n_cr, int n_ca, float *cr, float *ca,
                              float *ann, double *reg, cudaStream_t s) {
  if (n_pop > 0) unpack_population_kernel<<<n_pop, 256, 0, s>>>(z, n_par, n_cr, n_ca, cr, ca, ann, reg);
}

void launch_population_tiles(int n_pop, const float *ann, int n_ann, int H, int D, int KP1, int NP1,
                             unsigned short *tiles, cudaStream_t s) {
  const long long n = (long long)n_pop * H * D;
  if (n > 0)
    population_tiles_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_pop, ann, n_ann, H, D, KP1, NP1, tiles);
}

void launch_population_loss(int members, int n_struct, const int *offsets, const double *e_struct,
                            const double *w_struct, const double *e_tar, const double *w_tar,
                            const double *partial_gather, int nb_gather, int N, const double *reg, int n_par,
                            const double *lambda, double *loss, cudaStream_t s) {
  if (members > 0)
    population_loss_kernel<<<members, 256, 0, s>>>(n_struct, offsets, e_struct, w_struct, e_tar, w_tar,
                                                    partial_gather, nb_gather, N, reg, n_par, lambda[0], lambda[1],
                                                    lambda[2], lambda[3], lambda[4], loss);
}

void launch_struct_ids(int n_struct, const int *offsets, int *sid, cudaStream_t s) {
  if (n_struct > 0) struct_ids_kernel<<<n_struct, 128, 0, s>>>(n_struct, offsets, sid);
}

void launch_shift_tables(int n_struct, const Grid *grids, int ncode, int obits, float4 *dtab, cudaStream_t s) {
  const long long n = (long long)n_struct * ncode;
  if (n > 0) shift_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_struct, grids, ncode, obits, dtab);
}

void launch_struct_sums(int n_struct, int members, const int *offsets, int N, const double *e_atom,
                        const double *w_atom, double *e_struct, double *w_struct, int max_atoms, cudaStream_t s) {
  const long long units = (long long)n_struct * members;
  if (units > 0) {
    struct_sums_kernel<false><<<(unsigned)((units * 32 + 255) / 256), 256, 0, s>>>(n_struct, members, offsets, N,
                                                                                    e_atom, w_atom, e_struct, w_struct);
    if (max_atoms > kWideSum)
      struct_sums_kernel<true><<<(unsigned)units, kSumThreads, 0, s>>>(n_struct, members, offsets, N, e_atom, w_atom,
                                                                      e_struct, w_struct);
  }
}

// ------------------------------------------------------------------ host launchers
cudaError_t launch_rebuild(int N, int T, const Grid &g, const Batch &B, const float4 *dtab, float rlR2, float rlA2,
                           float rcR2, float rcA2, const AtomState &a, const ListBufs &L, int count_only,
                           BuildStatus *st, cudaStream_t s) {
  const int tb = 256;
  const int nb = (N + tb - 1) / tb;
  const int cb = (g.ncell + tb - 1) / tb;
  zero_cells_kernel<<<cb < 1024 ? cb : 1024, tb, 0, s>>>(g.ncell, L.cell_count, L.cell_cursor, st);
  bin_atoms_kernel<<<nb, tb, 0, s>>>(N, T, a, L.cell_count, g, B, st);
  scan_cells_kernel<<<1, 1024, 0, s>>>(g.ncell, L.cell_count, L.cell_start, st);
  scatter_atoms_kernel<<<nb, tb, 0, s>>>(N, a.cell_of, L.cell_start, L.cell_cursor, L.cell_atoms, B, st);
  sort_cells_kernel<<<cb, tb, 0, s>>>(g.ncell, L.cell_start, L.cell_atoms, st);
  reorder_gather_kernel<<<nb, tb, 0, s>>>(N, L.cell_atoms, a, B, st);
  reorder_commit_kernel<<<nb, tb, 0, s>>>(N, a, g, B, st);
  auto lists = [&](auto kern) {
    kern<<<(N + 127) / 128, 128, 0, s>>>(N, a.posA, a.pos4, a.cell_of, L.cell_start, g, B, rlR2, rlA2, rcR2, rcA2, L,
                                         count_only, st);
  };
  switch (T) {
    case 1: lists(build_lists_kernel<1>); break;
    case 2: lists(build_lists_kernel<2>); break;
    case 3: lists(build_lists_kernel<3>); break;
    case 4: lists(build_lists_kernel<4>); break;
    case 5: lists(build_lists_kernel<5>); break;
    case 6: lists(build_lists_kernel<6>); break;
    case 7: lists(build_lists_kernel<7>); break;
    default: lists(build_lists_kernel<8>); break;
  }
  if (!count_only) build_rev_kernel<<<nb, tb, 0, s>>>(N, L, g, B, st);
  if (B.sflag && B.n > 0) {
    const int sb = (B.n + 255) / 256;
    clear_sflags_kernel<<<sb < 256 ? sb : 256, 256, 0, s>>>(B.n, B.sflag, st);
  }
  finish_build_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

void launch_rebuild_condition(cudaGraphConditionalHandle hc, const BuildStatus *st, cudaStream_t s) {
  rebuild_condition_kernel<<<1, 1, 0, s>>>(hc, st);
}

void launch_iota(int N, int *perm, cudaStream_t s) { iota_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, perm); }

void launch_drift(int N, const AtomState &a, const double *inv_mass_kappa, double dt, double half_skin2,
                  BuildStatus *st, cudaStream_t s, const FireState *fire) {
  md_drift_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, a, inv_mass_kappa, dt, half_skin2, st, fire);
}

// FIRE velocity mixing after a velocity-Verlet step (Bitzek et al. 2006), one block, FP64
// sums in a fixed order: P = F . v, |F|, |v| over all atoms and max_i |F_i|^2. Converged
// when max_i |F_i| < fmax (then nothing moves again). Otherwise, for P > 0:
// v <- (1 - alpha) v + alpha |v| F / |F|, and after more than N_min such steps in a row the
// step grows (dt <- min(f_inc dt, dt_max)) and alpha shrinks (alpha <- f_alpha alpha); for
// P <= 0: v <- 0, dt <- f_dec dt, alpha <- alpha_start. check_only: only the convergence test
// (for the starting forces).
constexpr int kFireNmin = 5;
constexpr double kFireFinc = 1.1, kFireFdec = 0.5, kFireAlphaStart = 0.1, kFireFalpha = 0.99;

__global__ void fire_mix_kernel(int N, AtomState a, FireState *fire, int check_only) {
  __shared__ double red[4][1024];
  __shared__ int decision;
  if (fire->converged) return;
  double p = 0.0, ff = 0.0, vv = 0.0, fm = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double *F = a.F + 3 * (size_t)i, *v = a.v + 3 * (size_t)i;
    const double f2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    p += F[0] * v[0] + F[1] * v[1] + F[2] * v[2];
    ff += f2;
    vv += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    fm = fmax(fm, f2);
  }
  red[0][threadIdx.x] = p;
  red[1][threadIdx.x] = ff;
  red[2][threadIdx.x] = vv;
  red[3][threadIdx.x] = fm;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
      red[2][threadIdx.x] += red[2][threadIdx.x + o];
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  const double P = red[0][0], FF = red[1][0], VV = red[2][0], FM = red[3][0];
  if (threadIdx.x == 0) {
    decision = 0;
    if (!check_only) fire->steps += 1;  // velocity-Verlet steps taken
    if (FM < fire->fmax2) fire->converged = 1;
    else if (!check_only) decision = P > 0.0 ? 1 : 2;
  }
  __syncthreads();
  if (decision == 0) return;
  const double alpha = fire->alpha;
  const double c1 = decision == 1 ? 1.0 - alpha : 0.0;
  const double c2 = (decision == 1 && FF > 0.0) ? alpha * sqrt(VV / FF) : 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double *v = a.v + 3 * (size_t)i;
    const double *F = a.F + 3 * (size_t)i;
    for (int b = 0; b < 3; ++b) v[b] = c1 * v[b] + c2 * F[b];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (decision == 1) {
      if (fire->n_pos > kFireNmin) {
        fire->dt = fmin(fire->dt * kFireFinc, fire->dt_max);
        fire->alpha = alpha * kFireFalpha;
      }
      fire->n_pos += 1;
    } else {
      fire->dt *= kFireFdec;
      fire->alpha = kFireAlphaStart;
      fire->n_pos = 0;
    }
  }
}

void launch_fire_mix(int N, const AtomState &a, FireState *fire, int check_only, cudaStream_t s) {
  fire_mix_kernel<<<1, 1024, 0, s>>>(N, a, fire, check_only);
}

// ------------------------------------------------------------------ batched serving engine
// Every job is one structure of a batch; one iteration advances all of them together. The
// first iteration of a job only evaluates its forces (phase 0); each later one is a velocity-
// Verlet step (phase 1) of the job's own length (NVE) or FIRE step; finished jobs stay frozen.

// First half of the velocity-Verlet step of the stepping jobs: v += dt/2 F/m, x += dt v.
// A neighbour build is requested when an atom moved more than skin/2 since the last one.
__global__ void engine_drift_kernel(int N, AtomState a, const int *sid, const EngineSlot *slots,
                                    const double *inv_mass_kappa, double half_skin2, int *sflag, BuildStatus *st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const EngineSlot &sl = slots[sid[i]];
  if (sl.phase != 1 || sl.kind == kJobSingle || (sl.kind == kJobFire && sl.fire.converged)) return;
  const double dt = sl.kind == kJobFire ? sl.fire.dt : sl.dt;
  const double s = 0.5 * dt * inv_mass_kappa[a.types[i]];
  double d2 = 0.0, r[3];
  for (int b = 0; b < 3; ++b) {
    const size_t k = 3 * (size_t)i + b;
    const double vb = a.v[k] + s * a.F[k];
    a.v[k] = vb;
    r[b] = a.x[k] + dt * vb;
    a.x[k] = r[b];
    const double dd = r[b] - a.x_ref[k];
    d2 += dd * dd;
  }
  // the force kernels read the cell-local FP32 coordinates
  float4 p = a.pos4[i];
  p.x = (float)(r[0] - a.origin[3 * (size_t)i]);
  p.y = (float)(r[1] - a.origin[3 * (size_t)i + 1]);
  p.z = (float)(r[2] - a.origin[3 * (size_t)i + 2]);
  a.pos4[i] = p;
  // a build of this structure (also for a non-finite displacement, which the build reports)
  if (!(d2 <= half_skin2)) {
    if (sflag) sflag[sid[i]] = 1;
    st->rebuild = 1;
  }
}

// Clears the error flags of a chunk of iterations (a build is not requested).
__global__ void clear_flags_kernel(BuildStatus *st) {
  st->overflow = 0;
  st->rev_missing = 0;
  st->bad_input = 0;
  st->tc_timeout = 0;
}

void launch_clear_flags(BuildStatus *st, cudaStream_t s) { clear_flags_kernel<<<1, 1, 0, s>>>(st); }

// FIRE update of every FIRE job after its step (the FIRE definition of fire_mix_kernel, one
// block per job over the job's own atoms [offsets[s], offsets[s+1])); at the job's first
// iteration only the convergence test on the starting forces.
__global__ void engine_fire_kernel(const int *offsets, AtomState a, EngineSlot *slots) {
  const int s = blockIdx.x;
  EngineSlot &sl = slots[s];
  if (sl.kind != kJobFire || sl.phase == 2 || sl.fire.converged) return;
  const bool check_only = sl.phase == 0;
  __shared__ double red[4][256];
  __shared__ int decision;
  const int b0 = offsets[s], b1 = offsets[s + 1];
  double p = 0.0, ff = 0.0, vv = 0.0, fm = 0.0;
  for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const double *F = a.F + 3 * (size_t)i, *v = a.v + 3 * (size_t)i;
    const double f2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    p += F[0] * v[0] + F[1] * v[1] + F[2] * v[2];
    ff += f2;
    vv += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    fm = fmax(fm, f2);
  }
  red[0][threadIdx.x] = p;
  red[1][threadIdx.x] = ff;
  red[2][threadIdx.x] = vv;
  red[3][threadIdx.x] = fm;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
      red[2][threadIdx.x] += red[2][threadIdx.x + o];
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  const double P = red[0][0], FF = red[1][0], VV = red[2][0], FM = red[3][0];
  if (threadIdx.x == 0) {
    decision = 0;
    if (FM < sl.fire.fmax2) sl.fire.converged = 1;
    else if (!check_only) decision = P > 0.0 ? 1 : 2;
  }
  __syncthreads();
  if (decision == 0) return;
  const double alpha = sl.fire.alpha;
  const double c1 = decision == 1 ? 1.0 - alpha : 0.0;
  const double c2 = (decision == 1 && FF > 0.0) ? alpha * sqrt(VV / FF) : 0.0;
  for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    double *v = a.v + 3 * (size_t)i;
    const double *F = a.F + 3 * (size_t)i;
    for (int b = 0; b < 3; ++b) v[b] = c1 * v[b] + c2 * F[b];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (decision == 1) {
      if (sl.fire.n_pos > kFireNmin) {
        sl.fire.dt = fmin(sl.fire.dt * kFireFinc, sl.fire.dt_max);
        sl.fire.alpha = alpha * kFireFalpha;
      }
      sl.fire.n_pos += 1;
    } else {
      sl.fire.dt *= kFireFdec;
      sl.fire.alpha = kFireAlphaStart;
      sl.fire.n_pos = 0;
    }
  }
}

// Phase and step bookkeeping of every job after an iteration.
__global__ void engine_advance_kernel(int n_struct, EngineSlot *slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_struct) return;
  EngineSlot &sl = slots[s];
  const bool converged = sl.kind == kJobFire && sl.fire.converged;
  if (sl.phase == 0) {
    sl.phase = (sl.kind == kJobSingle || sl.n_steps <= 0 || converged) ? 2 : 1;
  } else if (sl.phase == 1) {
    sl.steps_done += 1;
    if (sl.steps_done >= sl.n_steps || converged) sl.phase = 2;
  }
}

// Move the atoms of the kept jobs to their new ranges: table[k] = (from, to, count, index
// shift of perm); one block per job.
__global__ void engine_relayout_kernel(const int4 *table, AtomState src, AtomState dst) {
  const int4 t = table[blockIdx.x];
  for (int k = threadIdx.x; k < t.z; k += blockDim.x) {
    const size_t i = (size_t)t.x + k, o = (size_t)t.y + k;
    for (int b = 0; b < 3; ++b) {
      dst.x[3 * o + b] = src.x[3 * i + b];
      dst.v[3 * o + b] = src.v[3 * i + b];
      dst.F[3 * o + b] = src.F[3 * i + b];
    }
    dst.types[o] = src.types[i];
    dst.perm[o] = src.perm[i] + t.w;
  }
}

void launch_engine_drift(int N, const AtomState &a, const int *sid, const EngineSlot *slots,
                         const double *inv_mass_kappa, double half_skin2, int *sflag, BuildStatus *st,
                         cudaStream_t s) {
  if (N > 0)
    engine_drift_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, a, sid, slots, inv_mass_kappa, half_skin2, sflag, st);
}

void launch_engine_fire(int n_struct, const int *offsets, const AtomState &a, EngineSlot *slots, cudaStream_t s) {
  if (n_struct > 0) engine_fire_kernel<<<n_struct, 256, 0, s>>>(offsets, a, slots);
}

void launch_engine_advance(int n_struct, EngineSlot *slots, cudaStream_t s) {
  if (n_struct > 0) engine_advance_kernel<<<(n_struct + 127) / 128, 128, 0, s>>>(n_struct, slots);
}

void launch_engine_relayout(int n_keep, const int4 *table, const AtomState &src, AtomState dst, cudaStream_t s) {
  if (n_keep > 0) engine_relayout_kernel<<<n_keep, 256, 0, s>>>(table, src, dst);
}

// Neighbour lists of internal atom i written to row perm[i] (the caller's order): the caller
// index of every neighbour and the FP32 pair vector the kernels use (cell-local coordinates
// plus the image shift). Radial lists are the per-type groups in type order.
__global__ void export_lists_kernel(int N, int T, const float4 *pos4, const int *perm, const ListBufs L,
                                    const float4 *dtab, int ncode, int jbits, unsigned jmask, int cap,
                                    int *nn_r, int *j_r, float *d_r, int *nn_a, int *j_a, float *d_a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 pi = pos4[i];
  const float4 *tab = dtab + (size_t)struct_of(pi) * ncode;  // structure 0 for a single structure
  const size_t row = (size_t)perm[i];
  int cnt = 0;
  for (int t = 0; t < T; ++t) cnt += L.nn_r[(size_t)t * N + i];
  nn_r[row] = cnt;
  for (int m = 0; m < cnt && m < cap && m < L.cap_r; ++m) {
    const unsigned e = L.nl_r[(size_t)m * N + i];
    const unsigned j = e & jmask;
    const float3 d = pair_vector(pi, pos4[j], tab[e >> jbits]);
    j_r[row * cap + m] = perm[j];
    d_r[(row * cap + m) * 3] = d.x;
    d_r[(row * cap + m) * 3 + 1] = d.y;
    d_r[(row * cap + m) * 3 + 2] = d.z;
  }
  const int na = L.nn_a[i];
  nn_a[row] = na;
  for (int m = 0; m < na && m < cap && m < L.cap_a; ++m) {
    const unsigned e = L.nl_a[(size_t)m * N + i];
    const unsigned j = e & jmask;
    const float3 d = pair_vector(pi, pos4[j], tab[e >> jbits]);
    j_a[row * cap + m] = perm[j];
    d_a[(row * cap + m) * 3] = d.x;
    d_a[(row * cap + m) * 3 + 1] = d.y;
    d_a[(row * cap + m) * 3 + 2] = d.z;
  }
}

void launch_export_lists(int N, int T, const float4 *pos4, const int *perm, const ListBufs &L, const float4 *dtab,
                         int ncode, int jbits, unsigned jmask, int cap, int *nn_r, int *j_r, float *d_r,
                         int *nn_a, int *j_a, float *d_a, cudaStream_t s) {
  export_lists_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, T, pos4, perm, L, dtab, ncode, jbits, jmask, cap,
                                                       nn_r, j_r, d_r, nn_a, j_a, d_a);
}

void launch_export(int N, const AtomState &a, const Grid &g, const Batch &B, double *pos, double *vel, double *force,
                   cudaStream_t s) {
  export_state_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, a, g, B, pos, vel, force);
}

void launch_finalize(int nb_atom, const double *partial_atom, int nb_gather, const double *partial_gather,
                     double *energy_total, double *virial_total, double *heat_total, double *thermo_stage,
                     int *thermo_ctl, int N, double volume, const ThermoState *ts, cudaStream_t s) {
  finalize_kernel<<<1, 256, 0, s>>>(nb_atom, partial_atom, nb_gather, partial_gather, energy_total, virial_total,
                                    heat_total, thermo_stage, thermo_ctl, N, volume, ts);
}

}  // namespace nep
