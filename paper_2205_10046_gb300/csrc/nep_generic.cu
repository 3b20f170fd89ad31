// NEP3 per-atom and gather kernels for any model shape, taken at run time.
//
// The compiled instantiations (nep_shape_*.cu) cover the workload shapes with every loop
// bound known to the compiler; this unit serves every other shape the parameters allow
// (n_max and N_bas up to 19, up to 256 neurons, l_max^3b 1..4, l_max^4b 0/2, l_max^5b 0/1),
// including the models the paper trains (Sec. III: MgAlCu n_max 12/8, carbon 10/8 with 100
// neurons). The arithmetic is the same (Eqs. qin, S_nk, the C3b/C4b/C5b forms, Ui, the
// partial forces and the gather of Eqs. F_ij, F_i, virial; Algorithms 1-4 fused into two
// kernels as in the compiled form), with run-time loops, the weights read from global
// memory, and per-thread arrays in local memory. FP32 network only.
#include <cuda_runtime.h>

#include "nep_kernels.cuh"

namespace nep {
namespace {

constexpr int kGenS = (kGenMaxN + 1) * 24;  // S_nk (then dU/dS_nk) of one atom

// f_k(r) for k = 0..K (Eq. f_n with the cosine cutoff), and f_k'(r) when fp is given.
__device__ __forceinline__ void basis_rt(float r, float inv_rc, int K, float *f, float *fp) {
  const float u = r * inv_rc;
  float sn, cs;
  __sincosf(3.14159265358979f * u, &sn, &cs);
  const float hfc = 0.25f * (1.f + cs), hfcp = -0.25f * 3.14159265358979f * inv_rc * sn;
  const float t1 = u - 1.f;
  const float x = 2.f * t1 * t1 - 1.f, xp = 4.f * t1 * inv_rc;
  float tkm1 = 1.f, tk = x, dkm1 = 0.f, dk = 1.f;
  f[0] = 2.f * hfc;
  if (fp) fp[0] = 2.f * hfcp;
  if (K >= 1) {
    f[1] = (x + 1.f) * hfc;
    if (fp) fp[1] = xp * hfc + (x + 1.f) * hfcp;
  }
  for (int k = 2; k <= K; ++k) {
    const float tn = 2.f * x * tk - tkm1;
    const float dn = 2.f * x * dk + 2.f * tk - dkm1;
    tkm1 = tk;
    tk = tn;
    dkm1 = dk;
    dk = dn;
    f[k] = (tn + 1.f) * hfc;
    if (fp) fp[k] = xp * dn * hfc + (tn + 1.f) * hfcp;
  }
}

// last polynomial index + 1 used by the 3-body terms and the 4-body term
__device__ __forceinline__ int n_poly(int L3, int L4) {
  const int k3 = L3 == 1 ? 3 : L3 == 2 ? 8 : L3 == 3 ? 15 : 24;
  return (L4 >= 2 && k3 < 8) ? 8 : k3;
}

template <bool DESC_ONLY, bool BATCH>
__global__ void __launch_bounds__(128) generic_atom_kernel(const AtomArgs a, const ModelF mf) {
  const int N = a.N, T = a.T;
  const int nR = a.gR, KR = a.gKR, nA = a.gA, KA = a.gKA, H = a.gH, L3 = a.gL3, L4 = a.gL4, L5 = a.gL5, D = a.gD;
  const int NK = n_poly(L3, L4);
  const int off4 = (nR + 1) + (nA + 1) * L3, off5 = off4 + (L4 >= 2 ? nA + 1 : 0);
  const int mem = BATCH ? (int)blockIdx.y : 0;
  const float *ann = (BATCH && a.pop_ann) ? a.pop_ann + mem * a.s_ann : a.ann;
  const float *w0 = ann, *b0 = ann + H * D, *w1 = b0 + H;
  const float b1 = w1[H];
  const float *c_r = a.c_r + mem * a.s_cr, *c_a = a.c_a + mem * a.s_ca;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double Ublock = 0.0;
  // (serving engine) atoms of a finished job frozen in the batch are skipped
  if (i < N && !(BATCH && a.slots && a.slots[struct_of(a.pos4[i])].phase == 2)) {
    const float4 pi = a.pos4[i];
    const int ti = type_of(pi);
    const float4 *tab = a.dtab + (BATCH ? (size_t)struct_of(pi) * a.ncode : 0);
    const float inv_rcR = 1.f / a.rcR, inv_rcA = 1.f / a.rcA;
    const float rcR2 = a.rcR * a.rcR, rcA2 = a.rcA * a.rcA;
    float q[kGenMaxDes];   // descriptor, then dU/dq
    float SD[kGenS];       // S_nk, then dU/dS_nk, row n at n * 24
    float f[kGenMaxN + 1], fp[kGenMaxN + 1], g[kGenMaxN + 1], gp[kGenMaxN + 1];
    for (int v = 0; v < D; ++v) q[v] = 0.f;
    for (int v = 0; v < (nA + 1) * 24; ++v) SD[v] = 0.f;
    // radial descriptor (Eq. qin), all neighbour types in one pass
    int cnt_r = 0;
    for (int t = 0; t < T; ++t) cnt_r += a.nn_r[(size_t)t * N + i];
    for (int m = 0; m < cnt_r; ++m) {
      const unsigned e = a.nl_r[(size_t)m * N + i];
      const float4 pj = a.pos4[e & a.jmask];
      const float3 d = pair_vector(pi, pj, tab[e >> a.jbits]);
      const float r2 = norm2(d);
      if (!(r2 < rcR2)) continue;
      basis_rt(sqrtf(r2), inv_rcR, KR, f, nullptr);
      const float *c = c_r + (size_t)(ti * T + type_of(pj)) * (nR + 1) * (KR + 1);
      for (int n = 0; n <= nR; ++n) {
        float acc = 0.f;
        for (int k = 0; k <= KR; ++k) acc = fmaf(c[n * (KR + 1) + k], f[k], acc);
        q[n] += acc;
      }
    }
    // angular sums S_nk (Eq. S_nk, b_k(d) r^-l)
    const int na = a.nn_a[i];
    for (int m = 0; m < na; ++m) {
      const unsigned e = a.nl_a[(size_t)m * N + i];
      const float4 pj = a.pos4[e & a.jmask];
      const float3 d = pair_vector(pi, pj, tab[e >> a.jbits]);
      const float r2 = norm2(d);
      if (!(r2 < rcA2)) continue;
      const float rinv = rsqrtf(r2);
      basis_rt(r2 * rinv, inv_rcA, KA, f, nullptr);
      const float *c = c_a + (size_t)(ti * T + type_of(pj)) * (nA + 1) * (KA + 1);
      for (int n = 0; n <= nA; ++n) {
        float acc = 0.f;
        for (int k = 0; k <= KA; ++k) acc = fmaf(c[n * (KA + 1) + k], f[k], acc);
        g[n] = acc;
      }
      const float rl[5] = {1.f, rinv, rinv * rinv, rinv * rinv * rinv, (rinv * rinv) * (rinv * rinv)};
      static_for<0, 24>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if (k < NK) {
          const float b = poly_b<k>(d.x, d.y, d.z, r2) * rl[l_of_k(k)];
          for (int n = 0; n <= nA; ++n) SD[n * 24 + k] = fmaf(g[n], b, SD[n * 24 + k]);
        }
      });
    }
    // angular descriptor components (Sec. II D)
    const int kend[5] = {0, 3, 8, 15, 24};
    for (int n = 0; n <= nA; ++n) {
      const float *s = SD + n * 24;
      for (int l = 1; l <= L3; ++l) {
        float acc = 0.f;
        for (int k = kend[l - 1]; k < kend[l]; ++k) acc = fmaf(mf.c3b[k] * s[k], s[k], acc);
        q[(nR + 1) + (l - 1) * (nA + 1) + n] = acc;
      }
      if (L4 >= 2)
        q[off4 + n] = mf.c4b[0] * s[3] * s[3] * s[3] + mf.c4b[1] * s[3] * (s[4] * s[4] + s[5] * s[5]) +
                      mf.c4b[2] * s[3] * (s[6] * s[6] + s[7] * s[7]) + mf.c4b[3] * s[6] * (s[5] * s[5] - s[4] * s[4]) +
                      mf.c4b[4] * s[4] * s[5] * s[7];
      if (L5 >= 1) {
        const float s12 = s[1] * s[1] + s[2] * s[2];
        q[off5 + n] = mf.c5b[0] * s[0] * s[0] * s[0] * s[0] + mf.c5b[1] * s[0] * s[0] * s12 + mf.c5b[2] * s12 * s12;
      }
    }
    if constexpr (DESC_ONLY) {
      const size_t io = a.perm ? (size_t)a.perm[i] : (size_t)i;
      for (int v = 0; v < D; ++v) a.q_out[io * D + v] = (double)q[v];
    } else {
      // network (Eq. Ui) and dU/dq; q is overwritten by dU/dq
      float beta[kGenMaxNeu];
      float U = 0.f;
      for (int mu = 0; mu < H; ++mu) {
        float z = -b0[mu];
        for (int v = 0; v < D; ++v) z = fmaf(w0[mu * D + v], q[v], z);
        const float h = tanhf(z);
        U = fmaf(w1[mu], h, U);
        beta[mu] = w1[mu] * (1.f - h * h);
      }
      U -= b1;
      for (int v = 0; v < D; ++v) {
        float acc = 0.f;
        for (int mu = 0; mu < H; ++mu) acc = fmaf(beta[mu], w0[mu * D + v], acc);
        q[v] = acc;
      }
      if (a.energy) a.energy[mem * a.s_out + (a.perm ? a.perm[i] : i)] = (double)U;
      Ublock = (double)U;
      // radial force coefficients e^t_k = sum_n dU/dq_n c^{t_i t}_nk and their sum
      float *erow = a.e_rad + mem * a.s_erad + (size_t)i * T * a.est;
      for (int t = 0; t < T; ++t) {
        const float *c = c_r + (size_t)(ti * T + t) * (nR + 1) * (KR + 1);
        float tot = 0.f;
        for (int k = 0; k <= KR; ++k) {
          float acc = 0.f;
          for (int n = 0; n <= nR; ++n) acc = fmaf(q[n], c[n * (KR + 1) + k], acc);
          erow[t * a.est + k] = acc;
          tot += acc;
        }
        erow[t * a.est + KR + 1] = tot;
        for (int k = KR + 2; k < a.est; ++k) erow[t * a.est + k] = 0.f;
      }
      // dU/dS_nk from the explicit 3/4/5-body forms, row by row in place
      for (int n = 0; n <= nA; ++n) {
        float s[24], dS[24];
        for (int k = 0; k < 24; ++k) s[k] = SD[n * 24 + k];
        for (int k = 0; k < 24; ++k) {
          const int l = l_of_k(k);
          dS[k] = (k < NK && l <= L3) ? 2.f * mf.c3b[k] * s[k] * q[(nR + 1) + (l - 1) * (nA + 1) + n] : 0.f;
        }
        if (L4 >= 2) {
          const float d4 = q[off4 + n];
          const float *C = mf.c4b;
          dS[3] += d4 * (3.f * C[0] * s[3] * s[3] + C[1] * (s[4] * s[4] + s[5] * s[5]) + C[2] * (s[6] * s[6] + s[7] * s[7]));
          dS[4] += d4 * (2.f * C[1] * s[3] * s[4] - 2.f * C[3] * s[6] * s[4] + C[4] * s[5] * s[7]);
          dS[5] += d4 * (2.f * C[1] * s[3] * s[5] + 2.f * C[3] * s[6] * s[5] + C[4] * s[4] * s[7]);
          dS[6] += d4 * (2.f * C[2] * s[3] * s[6] + C[3] * (s[5] * s[5] - s[4] * s[4]));
          dS[7] += d4 * (2.f * C[2] * s[3] * s[7] + C[4] * s[4] * s[5]);
        }
        if (L5 >= 1) {
          const float d5 = q[off5 + n];
          const float *C = mf.c5b;
          const float s12 = s[1] * s[1] + s[2] * s[2];
          dS[0] += d5 * (4.f * C[0] * s[0] * s[0] * s[0] + 2.f * C[1] * s[0] * s12);
          const float common = 2.f * C[1] * s[0] * s[0] + 4.f * C[2] * s12;
          dS[1] += d5 * common * s[1];
          dS[2] += d5 * common * s[2];
        }
        for (int k = 0; k < 24; ++k) SD[n * 24 + k] = dS[k];
      }
      // angular partial forces dU_i/dr_ij (angular terms of Eq. partial_force)
      float4 *pang = a.p_ang + mem * a.s_pang;
      for (int m = 0; m < na; ++m) {
        const unsigned e = a.nl_a[(size_t)m * N + i];
        const float4 pj = a.pos4[e & a.jmask];
        const float3 d = pair_vector(pi, pj, tab[e >> a.jbits]);
        const float r2 = norm2(d);
        if (!(r2 < rcA2)) continue;
        const float rinv = rsqrtf(r2);
        basis_rt(r2 * rinv, inv_rcA, KA, f, fp);
        const float *c = c_a + (size_t)(ti * T + type_of(pj)) * (nA + 1) * (KA + 1);
        for (int n = 0; n <= nA; ++n) {
          float acc = 0.f, accp = 0.f;
          for (int k = 0; k <= KA; ++k) {
            acc = fmaf(c[n * (KA + 1) + k], f[k], acc);
            accp = fmaf(c[n * (KA + 1) + k], fp[k], accp);
          }
          g[n] = acc;
          gp[n] = accp;
        }
        const float rl[5] = {1.f, rinv, rinv * rinv, rinv * rinv * rinv, (rinv * rinv) * (rinv * rinv)};
        float gx = 0.f, gy = 0.f, gz = 0.f, yy = 0.f;
        static_for<0, 24>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if (k < NK) {
            float ak = 0.f, ck = 0.f;
            for (int n = 0; n <= nA; ++n) {
              ak = fmaf(SD[n * 24 + k], g[n], ak);
              ck = fmaf(SD[n * 24 + k], gp[n], ck);
            }
            ak *= rl[l_of_k(k)];
            ck *= rl[l_of_k(k)];
            const float3 gb = poly_grad<k>(d.x, d.y, d.z, r2);
            gx = fmaf(ak, gb.x, gx);
            gy = fmaf(ak, gb.y, gy);
            gz = fmaf(ak, gb.z, gz);
            yy = fmaf(ck, poly_b<k>(d.x, d.y, d.z, r2), yy);
          }
        });
        const float ux = d.x * rinv, uy = d.y * rinv, uz = d.z * rinv;
        const float gu = gx * ux + gy * uy + gz * uz;
        pang[(size_t)m * N + i] =
            make_float4((gx - gu * ux) + yy * ux, (gy - gu * uy) + yy * uy, (gz - gu * uz) + yy * uz, 0.f);
      }
    }
  }
  if constexpr (!DESC_ONLY) {
    // deterministic block sum of U (fixed shuffle tree, then fixed warp order)
    __shared__ double red[4];
    double v = Ublock;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv];
      a.partial_atom[(size_t)mem * gridDim.x + blockIdx.x] = s;
    }
  }
}

// F_i and W_i (Algorithms 2 and 4, Eqs. F_ij, F_i, virial) with the run-time basis size of the
// radial coefficients; the epilogue (kick, kinetic energy, heat current, block sums) is the
// compiled gather kernel's.
template <bool BATCH>
__global__ void __launch_bounds__(128) generic_gather_kernel(const AtomArgs a) {
  const int mem = BATCH ? (int)blockIdx.y : 0;
  const float *e_rad = a.e_rad + mem * a.s_erad;
  const float4 *p_ang = a.p_ang + mem * a.s_pang;
  const int N = a.N, T = a.T, KR = a.gKR, est = a.est;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part[kReduceSlots];
  for (int s = 0; s < kReduceSlots; ++s) part[s] = 0.0;
  if (i < N && !(BATCH && a.slots && a.slots[struct_of(a.pos4[i])].phase == 2)) {
    const float4 pi = a.pos4[i];
    const int ti = type_of(pi);
    const float4 *tab = a.dtab + (BATCH ? (size_t)struct_of(pi) * a.ncode : 0);
    const float inv_rcR = 1.f / a.rcR;
    const float rcR2 = a.rcR * a.rcR, rcA2 = a.rcA * a.rcA;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float w[9];
    for (int c = 0; c < 9; ++c) w[c] = 0.f;
    int base = 0;
    for (int t = 0; t < T; ++t) {
      const int cnt = a.nn_r[(size_t)t * N + i];
      const float *eo = e_rad + ((size_t)i * T + t) * est;
      for (int m = base; m < base + cnt; ++m) {
        const unsigned e = a.nl_r[(size_t)m * N + i];
        const int j = e & a.jmask;
        const float3 d = pair_vector(pi, a.pos4[j], tab[e >> a.jbits]);
        const float r2 = norm2(d);
        if (!(r2 < rcR2)) continue;
        const float rinv = rsqrtf(r2);
        const float *ej = e_rad + ((size_t)j * T + ti) * est;
        float f[kGenMaxN + 1], fp[kGenMaxN + 1];
        basis_rt(r2 * rinv, inv_rcR, KR, f, fp);
        float si = 0.f, sj = 0.f;
        for (int k = 0; k <= KR; ++k) {
          si = fmaf(eo[k], fp[k], si);
          sj = fmaf(ej[k], fp[k], sj);
        }
        const float fs = (si + sj) * rinv;
        fx = fmaf(fs, d.x, fx);
        fy = fmaf(fs, d.y, fy);
        fz = fmaf(fs, d.z, fz);
        const float ws = -sj * rinv;
        const float px = ws * d.x, py = ws * d.y, pz = ws * d.z;
        w[0] = fmaf(d.x, px, w[0]); w[1] = fmaf(d.y, py, w[1]); w[2] = fmaf(d.z, pz, w[2]);
        w[3] = fmaf(d.x, py, w[3]); w[4] = fmaf(d.x, pz, w[4]); w[5] = fmaf(d.y, pz, w[5]);
        w[6] = fmaf(d.y, px, w[6]); w[7] = fmaf(d.z, px, w[7]); w[8] = fmaf(d.z, py, w[8]);
      }
      base += cnt;
    }
    const int na = a.nn_a[i];
    for (int m = 0; m < na; ++m) {
      const unsigned e = a.nl_a[(size_t)m * N + i];
      const float3 d = pair_vector(pi, a.pos4[e & a.jmask], tab[e >> a.jbits]);
      if (!(norm2(d) < rcA2)) continue;
      const float4 pij = p_ang[(size_t)m * N + i], pji = p_ang[a.rev_a[(size_t)m * N + i]];
      fx += pij.x - pji.x;
      fy += pij.y - pji.y;
      fz += pij.z - pji.z;
      w[0] = fmaf(d.x, pji.x, w[0]); w[1] = fmaf(d.y, pji.y, w[1]); w[2] = fmaf(d.z, pji.z, w[2]);
      w[3] = fmaf(d.x, pji.y, w[3]); w[4] = fmaf(d.x, pji.z, w[4]); w[5] = fmaf(d.y, pji.z, w[5]);
      w[6] = fmaf(d.y, pji.x, w[6]); w[7] = fmaf(d.z, pji.x, w[7]); w[8] = fmaf(d.z, pji.y, w[8]);
    }
    gather_epilogue(a, i, pi, ti, mem, fx, fy, fz, w, part);
  }
  gather_block_sums<128>(a, mem, part);
}

// ------------------------------------------------------------------------ launchers
cudaError_t generic_atom(const AtomArgs &a, const ModelF &mf, const float *, const float *, const float *, float,
                         int descriptor_only, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int blocks = (a.N + 127) / 128;
  if (descriptor_only) generic_atom_kernel<true, false><<<blocks, 128, 0, s>>>(a, mf);
  else generic_atom_kernel<false, false><<<blocks, 128, 0, s>>>(a, mf);
  return cudaGetLastError();
}

cudaError_t generic_gather(const AtomArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  generic_gather_kernel<false><<<(a.N + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// batches: one block shape (128 atoms per CTA), population members along grid.y
cudaError_t generic_atom_batch(const AtomArgs &a, const ModelF &mf, const float *, const float *, const float *,
                               float, int members, int block, cudaStream_t s) {
  if (a.N <= 0 || members <= 0) return cudaSuccess;
  if (block != 128 || a.precision != 0) return cudaErrorInvalidValue;
  generic_atom_kernel<false, true><<<dim3((a.N + 127) / 128, members), 128, 0, s>>>(a, mf);
  return cudaGetLastError();
}

cudaError_t generic_gather_batch(const AtomArgs &a, int members, int block, cudaStream_t s) {
  if (a.N <= 0 || members <= 0) return cudaSuccess;
  if (block != 128) return cudaErrorInvalidValue;
  generic_gather_kernel<true><<<dim3((a.N + 127) / 128, members), 128, 0, s>>>(a);
  return cudaGetLastError();
}

int blocks128(int N) { return (N + 127) / 128; }

}  // namespace

const ShapeOps *shape_generic() {
  static const ShapeOps ops = [] {
    ShapeOps o{};
    o.nR = o.KR = o.nA = o.KA = o.H = o.L3 = o.L4 = o.L5 = -1;  // any shape: taken from the handle
    o.n_des = 0;
    o.kp1 = o.np1 = 0;  // no tensor-core form
    o.atom = &generic_atom;
    o.gather = &generic_gather;
    o.atom_batch = &generic_atom_batch;
    o.gather_batch = &generic_gather_batch;
    o.atom_blocks = &blocks128;
    o.gather_blocks = &blocks128;
    o.lowreg = 0;
    return o;
  }();
  return &ops;
}

}  // namespace nep
