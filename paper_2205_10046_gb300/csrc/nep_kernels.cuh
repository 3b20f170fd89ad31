// NEP3 per-atom kernels for GB300 (sm_103a), templated on the model shape.
//
// Two kernels replace the four of the paper's Appendix B:
//   atom_kernel   one thread per atom: radial descriptor (Eq. qin), angular sums S_nk
//                 (Eq. S_nk) and the explicit 3/4/5-body components (Sec. II D), the
//                 network U_i and dU_i/dq (Eq. Ui), then the per-type radial force
//                 coefficients and the angular partial forces dU_i/dr_ij (the angular terms
//                 of Eq. partial_force), stored per angular pair (Algorithms 1 and 3 fused).
//   gather_kernel one thread per atom: F_i = sum_j [dU_i/dr_ij - dU_j/dr_ji] (Eqs. F_ij,
//                 F_i) and W_i = sum_j r_ij (x) dU_j/dr_ji (Eq. virial) for the radial
//                 part from both atoms' force coefficients and for the angular part from
//                 the stored partial forces of both atoms, with no atomics (Algorithms 2, 4).
//
// Differences from the paper's GPU design, for GB300:
//   * the radial descriptor accumulates the Chebyshev sums per neighbour type,
//     F^t_k = sum_{j of type t} f_k(r_ij), and contracts with c^{t_i t}_{nk} once per atom
//     (the radial list is grouped by neighbour type), so a pair costs O(K) instead of
//     O(n K); the radial partial forces likewise use e^t_k = sum_n dU/dq_n c^{t_i t}_{nk};
//   * S_nk are evaluated from the homogeneous polynomials b_k(d) scaled by r^-l, and the
//     angular gradient uses the tangential projection of grad b_k (no unit-vector round-off);
//   * pair vectors come from cell-local FP32 coordinates plus an image shift table, so no
//     FP64 arithmetic (slow on GB300) runs in the pair loops;
//   * all S_nk of an atom are summed in one pass in registers and wait in the thread's TMEM
//     lane while the network runs; dU/dS_nk stay in registers for the force loop (shapes
//     that do not fit fall back to passes over chunks of n and a shared-memory block).
#pragma once
#include <cuda_bf16.h>

#include <mutex>
#include <unordered_map>

#include "nep_internal.cuh"

namespace nep {

template <int NR_, int KR_, int NA_, int KA_, int H_, int L3_, int L4_, int L5_>
struct Shape {
  static constexpr int NR = NR_, KR = KR_, NA = NA_, KA = KA_, H = H_, L3 = L3_, L4 = L4_, L5 = L5_;
  static constexpr int NB = L3 + (L4 >= 2 ? 1 : 0) + (L5 >= 1 ? 1 : 0);
  static constexpr int NDES = (NR + 1) + (NA + 1) * NB;
  static constexpr int KEND3 = L3 == 1 ? 3 : L3 == 2 ? 8 : L3 == 3 ? 15 : 24;
  static constexpr int NK = KEND3 > 8 ? KEND3 : (L4 >= 2 ? 8 : KEND3);
  static constexpr int EST = ((KR + 2) + 3) / 4 * 4;  // KR+1 coefficients and their sum
  static constexpr int OFF4 = (NR + 1) + (NA + 1) * L3;
  static constexpr int OFF5 = OFF4 + (L4 >= 2 ? NA + 1 : 0);
  static constexpr int NDP = (NDES + 3) / 4 * 4;  // padded w0 row in shared memory
  // Shared-memory rows padded to whole float4s: c^A and c^R rows over k (KAP, KRP) and S_nk
  // rows over k (NKP). Without TMEM each thread parks its S_nk in a block of SPT floats,
  // n-major; SPT/4 is odd so the 16-byte accesses of 8 consecutive threads fall on 8 distinct
  // bank groups.
  static constexpr int KAP = (KA + 1 + 3) / 4 * 4;
  static constexpr int KRP = (KR + 1 + 3) / 4 * 4;  // c^R rows over k, padded likewise
  static constexpr int NKP = (NK + 3) / 4 * 4;
  static constexpr int SPT = ((NA + 1) * NKP / 4) % 2 ? (NA + 1) * NKP : (NA + 1) * NKP + 4;
  // float offsets of the shared regions after the shift table, each a whole number of float4s
  static constexpr int r4(int x) { return (x + 3) / 4 * 4; }
  static constexpr int off_b0(int prec) { return prec == 0 ? H * NDP : 0; }
  static constexpr int off_cR(int prec) { return off_b0(prec) + r4(2 * H); }
  static constexpr int off_cA(int prec, int T) { return off_cR(prec) + T * T * (NR + 1) * KRP; }
  static constexpr int off_S(int prec, int T) { return off_cA(prec, T) + T * T * (NA + 1) * KAP; }
  // S_nk is accumulated in NPASS passes over the angular neighbours, NCH values of n per
  // pass, so that at most ~4 x 24 accumulators are live at once
  static constexpr int NPASS = ((NA + 1) * NK > 144) ? ((NA + 1) + 3) / 4 : 1;
  static constexpr int NCH = ((NA + 1) + NPASS - 1) / NPASS;
  // tensor-core network (BF16 operands, FP32 accumulation in TMEM), one 128-atom tile:
  //   GEMM1 z[128 x NP1] = q[128 x KP1] . W0[NP1 x KP1]^T,  GEMM2 dq[128 x NP2] = beta[128 x KP2] . W0^T
  static constexpr int KP1 = (NDES + 15) / 16 * 16;
  static constexpr int NP1 = (H + 15) / 16 * 16;
  static constexpr int KP2 = NP1, NP2 = KP1;
  static constexpr int NS = (NA + 1) * NK;               // TMEM columns holding S_nk
  static constexpr int DCOL = (NS + 15) / 16 * 16;       // TMEM column of the GEMM results
  static constexpr int TMEM_COLS = 256;
  static constexpr int TILE_A = kAtomBlock * (KP1 > KP2 ? KP1 : KP2) * 2;  // bytes
  static constexpr int TILE_B = NP1 * KP1 * 2;                             // each of B1, B2
  static_assert(DCOL + (NP1 > NP2 ? NP1 : NP2) <= TMEM_COLS, "S and the network results must fit 256 TMEM columns");
  static_assert(NP1 <= 256 && NP2 <= 256, "UMMA N limit");
  // Low-register form of the tensor-core network: S_nk waits in the thread's shared block
  // (SPTC floats, later dU/dS_nk in place), the GEMM results take TMEM columns [0, ACOL) and
  // the A operands (BF16 pairs, one lane per atom) columns [ACOL, ACOL + KP/2): 128 columns a
  // block. With (SPTC/4) % 4 == 2 the rows are packed without padding and the float4 index is
  // rotated by ((thread >> 2) & 1), which keeps 8 consecutive threads on 8 distinct bank groups.
  // The split form keeps the A_lo operands after the A ones, at column ALO.
  static constexpr int ACOL = NP1 > NP2 ? NP1 : NP2;
  static constexpr int ALO = ACOL + (KP1 > KP2 ? KP1 : KP2) / 2;
  static constexpr bool TCLR_OK = NS <= 128 && NK % 8 == 0 && ALO <= 128;
  static constexpr bool TCLR2_OK = TCLR_OK && ALO + (KP1 > KP2 ? KP1 : KP2) / 2 <= 128;
  static constexpr int SW = (NA + 1) * NKP / 4;  // float4s of one thread's S_nk block
  static constexpr bool SROT = SW % 4 == 2;
  static constexpr int SPTC = SROT ? 4 * SW : SPT;
};

template <class S>
struct AnnConst {
  float w0[S::H * S::NDES];
  float b0[S::H];
  float w1[S::H];
  float b1;
  ModelF m;
};

// l of polynomial k (blocks 0-2, 3-7, 8-14, 15-23)
__host__ __device__ constexpr int l_of_k(int k) { return k < 3 ? 1 : k < 8 ? 2 : k < 15 ? 3 : 4; }

// b_k(d) of Sec. II D as homogeneous polynomials of the pair vector (s = |d|^2).
template <int k>
__device__ __forceinline__ float poly_b(float x, float y, float z, float s) {
  if constexpr (k == 0) return z;
  else if constexpr (k == 1) return x;
  else if constexpr (k == 2) return y;
  else if constexpr (k == 3) return 3.f * z * z - s;
  else if constexpr (k == 4) return x * z;
  else if constexpr (k == 5) return y * z;
  else if constexpr (k == 6) return x * x - y * y;
  else if constexpr (k == 7) return 2.f * x * y;
  else if constexpr (k == 8) return (5.f * z * z - 3.f * s) * z;
  else if constexpr (k == 9) return (5.f * z * z - s) * x;
  else if constexpr (k == 10) return (5.f * z * z - s) * y;
  else if constexpr (k == 11) return (x * x - y * y) * z;
  else if constexpr (k == 12) return 2.f * x * y * z;
  else if constexpr (k == 13) return (x * x - 3.f * y * y) * x;
  else if constexpr (k == 14) return (3.f * x * x - y * y) * y;
  else if constexpr (k == 15) return (35.f * z * z - 30.f * s) * z * z + 3.f * s * s;
  else if constexpr (k == 16) return (7.f * z * z - 3.f * s) * x * z;
  else if constexpr (k == 17) return (7.f * z * z - 3.f * s) * y * z;
  else if constexpr (k == 18) return (7.f * z * z - s) * (x * x - y * y);
  else if constexpr (k == 19) return (7.f * z * z - s) * 2.f * x * y;
  else if constexpr (k == 20) return (x * x - 3.f * y * y) * x * z;
  else if constexpr (k == 21) return (3.f * x * x - y * y) * y * z;
  else if constexpr (k == 22) return (x * x - y * y) * (x * x - y * y) - 4.f * x * x * y * y;
  else return 4.f * (x * x - y * y) * x * y;
}

// Gradient of b_k(d) with s = |d|^2 held fixed. Only its component tangential to d is
// used: grad |d|^2 = 2d is radial, so the tangential part equals that of the full gradient.
template <int k>
__device__ __forceinline__ float3 poly_grad(float x, float y, float z, float s) {
  if constexpr (k == 0) return make_float3(0.f, 0.f, 1.f);
  else if constexpr (k == 1) return make_float3(1.f, 0.f, 0.f);
  else if constexpr (k == 2) return make_float3(0.f, 1.f, 0.f);
  else if constexpr (k == 3) return make_float3(0.f, 0.f, 6.f * z);
  else if constexpr (k == 4) return make_float3(z, 0.f, x);
  else if constexpr (k == 5) return make_float3(0.f, z, y);
  else if constexpr (k == 6) return make_float3(2.f * x, -2.f * y, 0.f);
  else if constexpr (k == 7) return make_float3(2.f * y, 2.f * x, 0.f);
  else if constexpr (k == 8) return make_float3(0.f, 0.f, 15.f * z * z - 3.f * s);
  else if constexpr (k == 9) return make_float3(5.f * z * z - s, 0.f, 10.f * x * z);
  else if constexpr (k == 10) return make_float3(0.f, 5.f * z * z - s, 10.f * y * z);
  else if constexpr (k == 11) return make_float3(2.f * x * z, -2.f * y * z, x * x - y * y);
  else if constexpr (k == 12) return make_float3(2.f * y * z, 2.f * x * z, 2.f * x * y);
  else if constexpr (k == 13) return make_float3(3.f * (x * x - y * y), -6.f * x * y, 0.f);
  else if constexpr (k == 14) return make_float3(6.f * x * y, 3.f * (x * x - y * y), 0.f);
  else if constexpr (k == 15) return make_float3(0.f, 0.f, (140.f * z * z - 60.f * s) * z);
  else if constexpr (k == 16) return make_float3((7.f * z * z - 3.f * s) * z, 0.f, (21.f * z * z - 3.f * s) * x);
  else if constexpr (k == 17) return make_float3(0.f, (7.f * z * z - 3.f * s) * z, (21.f * z * z - 3.f * s) * y);
  else if constexpr (k == 18)
    return make_float3(2.f * x * (7.f * z * z - s), -2.f * y * (7.f * z * z - s), 14.f * z * (x * x - y * y));
  else if constexpr (k == 19)
    return make_float3(2.f * y * (7.f * z * z - s), 2.f * x * (7.f * z * z - s), 28.f * x * y * z);
  else if constexpr (k == 20)
    return make_float3(3.f * (x * x - y * y) * z, -6.f * x * y * z, (x * x - 3.f * y * y) * x);
  else if constexpr (k == 21)
    return make_float3(6.f * x * y * z, 3.f * (x * x - y * y) * z, (3.f * x * x - y * y) * y);
  else if constexpr (k == 22)
    return make_float3(4.f * x * (x * x - 3.f * y * y), 4.f * y * (y * y - 3.f * x * x), 0.f);
  else return make_float3(4.f * y * (3.f * x * x - y * y), 4.f * x * (x * x - 3.f * y * y), 0.f);
}

// Unrolled compile-time loop helper.
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// ------------------------------------------------------------------ tcgen05 / mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, LBO (next 8x16-byte core matrix
// along K), SBO (next core matrix along M/N), version bit.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with B read MN-major (transpose-B bit): core matrices of 8 K-rows x 16 bytes of
// consecutive N, SBO the step along N and LBO the step along K. A K-major tile of W0 for
// D = A.W0^T read this way is W0 itself as the K x N operand of D = A.W0.
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16_bmn() {
  return umma_idesc_bf16<M, N>() | (1u << 16);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

// Wait for an mbarrier phase with an iteration limit; returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}

// The same MMA with the A operand read from tensor memory (lane m = row m, K packed along the
// columns: two BF16 values per 32-bit column, the lower K index in the low half).
__device__ __forceinline__ void umma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc,
                                             uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&b);
}

// Byte offset of element (row r, k) in a K-major no-swizzle operand tile with KC = K/8
// 16-byte chunks per row group: core matrix (r/8, k/8) at ((r/8) KC + k/8) * 128.
__host__ __device__ constexpr int umma_off(int r, int k, int KC) {
  return ((r / 8) * KC + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// f_k(r) = (T_k(x) + 1) fc/2 with fc = (1 + cos(pi r/rc))/2 and x = 2(r/rc - 1)^2 - 1
// (Eq. f_n and the cosine cutoff); fills f[0..K].
template <int K>
__device__ __forceinline__ void cheb_basis(float r, float inv_rc, float *f) {
  const float u = r * inv_rc;
  const float hfc = 0.25f * (1.f + __cosf(3.14159265358979f * u));
  const float t1 = u - 1.f;
  const float x = 2.f * t1 * t1 - 1.f;
  const float x2 = 2.f * x;
  float tkm1 = 1.f, tk = x;
  f[0] = 2.f * hfc;
  if constexpr (K >= 1) f[1] = __fmaf_rn(x, hfc, hfc);
#pragma unroll
  for (int k = 2; k <= K; ++k) {
    const float tn = __fmaf_rn(x2, tk, -tkm1);
    tkm1 = tk;
    tk = tn;
    f[k] = __fmaf_rn(tn, hfc, hfc);
  }
}

// f_k(r) and f_k'(r) for k = 0..K.
template <int K>
__device__ __forceinline__ void cheb_basis_d(float r, float inv_rc, float *f, float *fp) {
  const float u = r * inv_rc;
  float sn, cs;
  __sincosf(3.14159265358979f * u, &sn, &cs);
  const float hfc = 0.25f * (1.f + cs);                       // fc/2
  const float hfcp = -0.25f * 3.14159265358979f * inv_rc * sn; // fc'/2
  const float t1 = u - 1.f;
  const float x = 2.f * t1 * t1 - 1.f;
  const float xp = 4.f * t1 * inv_rc;  // dx/dr
  const float x2 = 2.f * x;
  const float a = xp * hfc;            // T_k' coefficient
  float tkm1 = 1.f, tk = x, dkm1 = 0.f, dk = 1.f;
  f[0] = 2.f * hfc;
  fp[0] = 2.f * hfcp;
  if constexpr (K >= 1) {
    f[1] = __fmaf_rn(x, hfc, hfc);
    fp[1] = __fmaf_rn(a, 1.f, (x + 1.f) * hfcp);
  }
#pragma unroll
  for (int k = 2; k <= K; ++k) {
    const float tn = __fmaf_rn(x2, tk, -tkm1);
    const float dn = __fmaf_rn(x2, dk, __fmaf_rn(2.f, tk, -dkm1));
    tkm1 = tk;
    tk = tn;
    dkm1 = dk;
    dk = dn;
    f[k] = __fmaf_rn(tn, hfc, hfc);
    fp[k] = __fmaf_rn(a, dn, (tn + 1.f) * hfcp);
  }
}

// Loop over the cnt list entries of atom i starting at slot `slot0` (slot-major lists),
// software-pipelined: the list entry is fetched two iterations ahead and the neighbour's
// position one iteration ahead, so the gathers overlap the arithmetic of earlier pairs.
template <class Body>
__device__ __forceinline__ void for_pairs(const unsigned *__restrict__ nl, int slot0, int cnt, int N, int i,
                                          const float4 *__restrict__ pos4, unsigned jmask, Body &&body) {
  if (cnt <= 0) return;
  const unsigned *col = nl + (size_t)slot0 * N + i;
  unsigned e0 = __ldg(col);
  unsigned e1 = cnt > 1 ? __ldg(col + N) : 0u;
  float4 p0 = __ldg(pos4 + (e0 & jmask));
  for (int m = 0; m < cnt; ++m) {
    const unsigned e = e0;
    const float4 pj = p0;
    if (m + 1 < cnt) p0 = __ldg(pos4 + (e1 & jmask));
    e0 = e1;
    if (m + 2 < cnt) e1 = __ldg(col + (size_t)(m + 2) * N);
    body(m, e, pj);
  }
}

// Request the line holding *p into L2 (no register, no wait). Callers keep p inside the
// list allocation: slot rows below the list capacity.
__device__ __forceinline__ void l2_prefetch(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Load of a list entry: read-only cached, or streaming (evict-first) for a list that the
// kernel reads only once, so that it does not push the neighbours' data out of L1.
template <bool STREAM, class T>
__device__ __forceinline__ T ld_list(const T *p) {
  if constexpr (STREAM) return __ldcs(p);
  else return __ldg(p);
}

// Batched variant for short pair bodies: the positions of D pairs are requested together and
// the list entries AHEAD (1 or 2) batches ahead (the lists stream from DRAM).
template <int D, bool STREAM = false, int AHEAD = 2, class Body>
__device__ __forceinline__ void for_pairs_batch(const unsigned *__restrict__ nl, int slot0, int cnt, int N, int i,
                                                const float4 *__restrict__ pos4, unsigned jmask, Body &&body) {
  if (cnt <= 0) return;
  const unsigned *col = nl + (size_t)slot0 * N + i;
  unsigned e[D], en[D];
#pragma unroll
  for (int d = 0; d < D; ++d) e[d] = d < cnt ? ld_list<STREAM>(col + (size_t)d * N) : 0u;
  if constexpr (AHEAD == 2) {
#pragma unroll
    for (int d = 0; d < D; ++d) en[d] = D + d < cnt ? ld_list<STREAM>(col + (size_t)(D + d) * N) : 0u;
  }
  for (int m0 = 0; m0 < cnt; m0 += D) {
    float4 p[D];
#pragma unroll
    for (int d = 0; d < D; ++d) p[d] = __ldg(pos4 + (e[d] & jmask));
    unsigned enn[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int m = m0 + AHEAD * D + d;
      enn[d] = m < cnt ? ld_list<STREAM>(col + (size_t)m * N) : 0u;
    }
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (m0 + d < cnt) body(m0 + d, e[d], p[d]);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if constexpr (AHEAD == 2) {
        e[d] = en[d];
        en[d] = enn[d];
      } else {
        e[d] = enn[d];
      }
    }
  }
}

// Plain loop over list entries (for pair bodies long enough to hide the gather themselves).
template <class Body>
__device__ __forceinline__ void for_pairs_plain(const unsigned *__restrict__ nl, int cnt, int N, int i,
                                                const float4 *__restrict__ pos4, unsigned jmask, Body &&body) {
  for (int m = 0; m < cnt; ++m) {
    const unsigned e = __ldg(nl + (size_t)m * N + i);
    body(m, e, __ldg(pos4 + (e & jmask)));
  }
}

// ------------------------------------------------------------------------ per-atom kernel
// OCC = 3 is the low-register form of the FP32 kernel: S_nk summed in two passes over the
// angular neighbours, parked in 128 TMEM columns, and dU/dS_nk kept in the thread's shared
// block instead of registers, so that three blocks (12 warps) fit an SM instead of two.
template <class S, bool DESC_ONLY, int PREC, bool BATCH = false, int AB = kAtomBlock, int OCC = 1>
__global__ void __launch_bounds__(AB, OCC)
    atom_kernel(const AtomArgs a, const __grid_constant__ AnnConst<S> w) {
  static_assert(PREC >= 0 && PREC <= 2, "network forms: 0 FP32, 1 BF16, 2 split BF16");
  constexpr bool LOWREG = OCC > 1;
  static_assert(!LOWREG || (!DESC_ONLY && AB == 128 && S::NS <= 128 && S::NK % 8 == 0),
                "the low-register form: S_nk within 128 TMEM columns");
  // TCLR: the low-register form with a tensor-core network. S_nk then waits in the thread's
  // shared block (not in TMEM), whose 128 columns hold the GEMM operands and results.
  constexpr bool TCLR = LOWREG && PREC >= 1;
  static_assert(!TCLR || (PREC == 1 ? S::TCLR_OK : S::TCLR2_OK), "the tensor-core network within 128 TMEM columns");
  constexpr uint32_t TCOLS = LOWREG ? 128u : (uint32_t)S::TMEM_COLS;
  static_assert(PREC == 0 || !DESC_ONLY, "the descriptor-only kernel has no network");
  static_assert(PREC == 0 || AB == 128, "the tensor-core network works on 128-atom tiles (UMMA M = 128)");
  // S_nk waits for the network in this thread's TMEM lane (128-atom blocks, whole groups of 8
  // columns), else in a per-thread block of shared memory
  constexpr bool TM = !DESC_ONLY && AB == 128 && S::NK % 8 == 0;
  static_assert(PREC == 0 || TM, "the tensor-core network works in TMEM");
  constexpr bool STM = TM && !TCLR;  // S_nk parked in TMEM during the network
  // With S_nk parked in TMEM the registers hold all (n_max^A + 1) x 24 sums at once: one pass
  // over the angular neighbours (PbTe: 168 sums); otherwise NPASS passes of NCH values of n.
  constexpr int NPASS = LOWREG ? ((S::NA + 1) >= 2 ? 2 : 1) : (TM && (S::NA + 1) * S::NK <= 192 ? 1 : S::NPASS);
  constexpr int NCH = (S::NA + 1 + NPASS - 1) / NPASS;
  static_assert(AB % 32 == 0 && AB <= 256, "whole warps, at most 256 atoms per block");
  constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, NK = S::NK, NDES = S::NDES;
  extern __shared__ float4 smem4[];
  const int T = a.T;
  const int N = a.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // Threads past the last atom, and (serving engine) atoms of a finished job frozen in the
  // batch, run the same code with no neighbours (the tensor-core steps are block- and
  // warp-collective); they write nothing.
  // This atom's position, list lengths and first list entries are requested before the
  // block's setup (shared tables, TMEM), which hides their DRAM latency: the counts into
  // registers, the first 16 radial and 2 angular slots into L2.
  const float4 pi = i < N ? __ldg(a.pos4 + i) : make_float4(0.f, 0.f, 0.f, __int_as_float(0));
  const bool active = i < N && !(BATCH && a.slots && a.slots[struct_of(pi)].phase == 2);
  const int na = active ? __ldg(a.nn_a + i) : 0;
  int cnt_r = active ? __ldg(a.nn_r + i) : 0;
  if (active) {
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (m < a.cap_r) l2_prefetch(a.nl_r + (size_t)m * N + i);
#pragma unroll
    for (int m = 0; m < 2; ++m)
      if (m < a.cap_a) l2_prefetch(a.nl_a + (size_t)m * N + i);
  }
  constexpr int NDP = S::NDP;
  // batches: the shift tables stay in global memory, one per structure, and blockIdx.y is
  // the population member whose coefficients and network this block evaluates
  const int mem = BATCH ? (int)blockIdx.y : 0;
  const float *pw = (BATCH && a.pop_ann) ? a.pop_ann + mem * a.s_ann : nullptr;
  float4 *dtab_s = smem4;                                        // [ncode] (one structure)
  constexpr int KAP = S::KAP, NKP = S::NKP, SPT = TCLR ? S::SPTC : S::SPT;
  float *w0_s = reinterpret_cast<float *>(smem4 + (BATCH ? 0 : a.ncode));  // [H][NDP] (FP32 network)
  float *b0_s = w0_s + S::off_b0(PREC);                          // [H]
  float *w1_s = b0_s + S::H;                                     // [H]
  float *cR_s = w0_s + S::off_cR(PREC);                          // [T][T][NR+1][KRP]
  float *cA_s = w0_s + S::off_cA(PREC, T);                       // [T][T][NA+1][KAP]
  // [block][SPT]: each thread's S_nk ([n][NKP]) while the network runs (without TMEM), or
  // the BF16 operand tiles of the tensor-core network
  float *S_s = w0_s + S::off_S(PREC, T);
  if constexpr (!BATCH)
    for (int v = threadIdx.x; v < a.ncode; v += blockDim.x) dtab_s[v] = a.dtab[v];
  if constexpr (PREC == 0) {
    for (int v = threadIdx.x; v < S::H * NDP; v += blockDim.x) {
      const int mu = v / NDP, c = v - mu * NDP;
      w0_s[v] = c < NDES ? (pw ? pw[mu * NDES + c] : w.w0[mu * NDES + c]) : 0.f;
    }
  }
  for (int v = threadIdx.x; v < S::H; v += blockDim.x) {
    b0_s[v] = pw ? pw[S::H * NDES + v] : w.b0[v];
    w1_s[v] = pw ? pw[S::H * NDES + S::H + v] : w.w1[v];
  }
  __shared__ float b1_s;
  if (threadIdx.x == 0) b1_s = pw ? pw[S::H * NDES + 2 * S::H] : w.b1;
  const float *c_r = a.c_r + mem * a.s_cr, *c_a = a.c_a + mem * a.s_ca;
  constexpr int KRP = S::KRP;
  for (int v = threadIdx.x; v < T * T * (NR + 1) * KRP; v += blockDim.x) {
    const int row = v / KRP, k = v - row * KRP;
    cR_s[v] = k <= KR ? c_r[row * (KR + 1) + k] : 0.f;
  }
  for (int v = threadIdx.x; v < T * T * (NA + 1) * KAP; v += blockDim.x) {
    const int row = v / KAP, k = v - row * KAP;
    cA_s[v] = k <= KA ? c_a[row * (KA + 1) + k] : 0.f;
  }
  // tensor-core network: operand tiles (128-byte aligned) and TMEM for S_nk and the results
  __shared__ __align__(8) uint64_t tc_mbar;
  __shared__ uint32_t tc_tmem;
  // PREC 2 splits every operand value into two BF16 terms (hi + lo) and adds the products
  // hi.hi + lo.hi + hi.lo: operand tiles A_lo, B1_lo, B2_lo follow the plain ones
  constexpr bool SPLIT = PREC == 2;
  unsigned char *tileA = nullptr, *tileB1 = nullptr, *tileB2 = nullptr;
  unsigned char *tileAlo = nullptr, *tileB1lo = nullptr, *tileB2lo = nullptr;
  if constexpr (PREC >= 1) {
    // (TCLR: after the per-thread S_nk blocks, and no A tile: the A operands are in TMEM)
    unsigned char *base = reinterpret_cast<unsigned char *>(S_s + (TCLR ? AB * SPT : 0));
    base += (128u - (smem_addr(base) & 127u)) & 127u;
    tileA = base;
    tileB1 = tileA + (TCLR ? 0 : S::TILE_A);
    tileB2 = tileB1 + S::TILE_B;
    if constexpr (SPLIT) {
      tileB1lo = tileB2 + S::TILE_B;
      tileB2lo = tileB1lo + S::TILE_B;
      tileAlo = tileB2lo + S::TILE_B;
    }
    if constexpr (TCLR) {  // one W0 tile (and its lo part) serves both GEMMs
      tileB1lo = tileB1 + S::TILE_B;
      tileB2 = tileB2lo = tileA = tileAlo = nullptr;
    }
    // W0 tiles in global memory: B1, B2, then (split form) B1_lo, B2_lo
    const uint4 *b1t = a.tc_b1, *b2t = a.tc_b2;
    if (BATCH && a.pop_tc) {
      b1t = a.pop_tc + mem * a.s_tc;
      b2t = b1t + S::TILE_B / 16;
    }
    for (int v = threadIdx.x; v < S::TILE_B / 16; v += blockDim.x) {
      reinterpret_cast<uint4 *>(tileB1)[v] = b1t[v];
      if constexpr (!TCLR) reinterpret_cast<uint4 *>(tileB2)[v] = b2t[v];
      if constexpr (SPLIT) {
        reinterpret_cast<uint4 *>(tileB1lo)[v] = b1t[v + 2 * (S::TILE_B / 16)];
        if constexpr (!TCLR) reinterpret_cast<uint4 *>(tileB2lo)[v] = b2t[v + 2 * (S::TILE_B / 16)];
      }
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&tc_mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if constexpr (TM) {
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tc_tmem)),
                   "r"(TCOLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  uint32_t tmem_row = 0;  // TMEM address of this warp's 32 lanes, column 0
  if constexpr (TM) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_row = tc_tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
  }
  // this thread's shared block of S_nk, later dU/dS_nk: float4 v of [n][NKP / 4]
  float4 *const Sblk = reinterpret_cast<float4 *>(S_s + threadIdx.x * SPT);
  const int srot = (TCLR && S::SROT) ? ((threadIdx.x >> 2) & 1) : 0;
  auto sref = [&](int v) -> float4 & {
    if constexpr (TCLR && S::SROT) return v == S::SW - 1 ? Sblk[srot ? 0 : S::SW - 1] : Sblk[v + srot];
    else return Sblk[v];
  };

  double Ublock = 0.0;
  {
    const int ti = type_of(pi);
    const float inv_rcR = 1.f / a.rcR, inv_rcA = 1.f / a.rcA;
    const float rcR2 = a.rcR * a.rcR, rcA2 = a.rcA * a.rcA;
    // shift vector of a list entry: from shared memory, or from the structure's own table
    const float4 *dtab_b = BATCH ? a.dtab + (size_t)struct_of(pi) * a.ncode : dtab_s;
    auto shift = [&](unsigned e) -> float4 {
      if constexpr (BATCH) return __ldg(dtab_b + (e >> a.jbits));
      else return dtab_s[e >> a.jbits];
    };

    float q[NDES];
#pragma unroll
    for (int v = 0; v < NDES; ++v) q[v] = 0.f;

    // ---- radial descriptor, Eq. qin: per neighbour type, F^t_k = sum_j f_k(r_ij). With
    // f_k = (T_k(x) + 1) fc/2 the sums are kept as sum_j T_k(x_j) fc_j/2 (k >= 1) and
    // H = sum_j fc_j/2, added once at the end: F_0 = 2H, F_k = sum_j T_k fc_j/2 + H.
    int base = 0;
    for (int t = 0; t < T; ++t) {
      const int cnt = cnt_r;
      if (t + 1 < T) {  // the next type's count, and its first 16 slots into L2
        cnt_r = active ? __ldg(a.nn_r + (size_t)(t + 1) * N + i) : 0;
        if (active)
#pragma unroll
          for (int m = 0; m < 16; ++m)
            if (base + cnt + m < a.cap_r) l2_prefetch(a.nl_r + (size_t)(base + cnt + m) * N + i);
      }
      float Fk[KR + 1];
#pragma unroll
      for (int k = 0; k <= KR; ++k) Fk[k] = 0.f;
      for_pairs_batch<8, true>(a.nl_r, base, cnt, N, i, a.pos4, a.jmask, [&](int, unsigned e, const float4 &pj) {
        const float3 d = pair_vector(pi, pj, shift(e));
        const float r2 = norm2(d);
        if (r2 < rcR2) {
          const float u = r2 * rsqrtf(r2) * inv_rcR;
          const float hfc = 0.25f * (1.f + __cosf(3.14159265358979f * u));
          const float t1 = u - 1.f;
          const float x = 2.f * t1 * t1 - 1.f;
          const float x2 = 2.f * x;
          Fk[0] += hfc;
          if constexpr (KR >= 1) Fk[1] = __fmaf_rn(x, hfc, Fk[1]);
          float tkm1 = 1.f, tk = x;
#pragma unroll
          for (int k = 2; k <= KR; ++k) {
            const float tn = __fmaf_rn(x2, tk, -tkm1);
            tkm1 = tk;
            tk = tn;
            Fk[k] = __fmaf_rn(tn, hfc, Fk[k]);
          }
        }
      });
#pragma unroll
      for (int k = 1; k <= KR; ++k) Fk[k] += Fk[0];
      Fk[0] *= 2.f;
      const float4 *c = reinterpret_cast<const float4 *>(cR_s + (ti * T + t) * (NR + 1) * KRP);
#pragma unroll
      for (int n = 0; n <= NR; ++n) {
        float acc = q[n];
#pragma unroll
        for (int k4 = 0; k4 < KRP / 4; ++k4) {
          const float4 cv = c[n * (KRP / 4) + k4];
          const float cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (4 * k4 + j <= KR) acc = __fmaf_rn(cw[j], Fk[4 * k4 + j], acc);
        }
        q[n] = acc;
      }
      base += cnt;
    }

    // ---- angular sums S_nk (Eq. S_nk, b_k(d) r^-l) and the angular descriptor components
    // (Sec. II D): one pass over the angular neighbours, or one chunk of n per pass when the
    // sums do not fit the registers (NPASS above)
    if constexpr (LOWREG) {
      // low-register form: two passes split over k, pass 0 the polynomials k < 16 (the 3-body
      // blocks l = 1..3 and k = 15 of l = 4, the 4- and 5-body terms), pass 1 the rest; every
      // pass sums all n, so each pair evaluates each b_k once
      constexpr int KSPL = NK > 16 ? 16 : NK;
      static_for<0, (NK > KSPL ? 2 : 1)>([&](auto pc) {
        constexpr int k0 = decltype(pc)::value == 0 ? 0 : KSPL;
        constexpr int k1 = decltype(pc)::value == 0 ? KSPL : NK;
        constexpr int NKC = k1 - k0;
        float Sv[NA + 1][NKC];
#pragma unroll
        for (int n = 0; n <= NA; ++n)
#pragma unroll
          for (int k = 0; k < NKC; ++k) Sv[n][k] = 0.f;
        for_pairs(a.nl_a, 0, na, N, i, a.pos4, a.jmask, [&](int, unsigned e, const float4 &pj) {
          const float3 d = pair_vector(pi, pj, shift(e));
          const float r2 = norm2(d);
          if (r2 < rcA2) {
            const int tj = type_of(pj);
            const float rinv = rsqrtf(r2);
            float f[KA + 1];
            cheb_basis<KA>(r2 * rinv, inv_rcA, f);
            const float4 *cc = reinterpret_cast<const float4 *>(cA_s + (ti * T + tj) * (NA + 1) * KAP);
            float g[NA + 1];
#pragma unroll
            for (int n = 0; n <= NA; ++n) {
              float acc = 0.f;
#pragma unroll
              for (int k4 = 0; k4 < KAP / 4; ++k4) {
                const float4 cv = cc[n * (KAP / 4) + k4];
                const float cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  if (4 * k4 + j <= KA) acc = __fmaf_rn(cw[j], f[4 * k4 + j], acc);
              }
              g[n] = acc;
            }
            const float rl[5] = {1.f, rinv, rinv * rinv, rinv * rinv * rinv, (rinv * rinv) * (rinv * rinv)};
            static_for<k0, k1>([&](auto kc) {
              constexpr int k = decltype(kc)::value;
              const float b = poly_b<k>(d.x, d.y, d.z, r2) * rl[l_of_k(k)];
#pragma unroll
              for (int n = 0; n <= NA; ++n) Sv[n][k - k0] = __fmaf_rn(g[n], b, Sv[n][k - k0]);
            });
          }
        });
#pragma unroll
        for (int n = 0; n <= NA; ++n) {
          // 3-body components: the part of each l block inside [k0, k1)
          static_for<0, S::L3>([&](auto lc) {
            constexpr int l = decltype(lc)::value + 1;
            constexpr int b0 = l == 1 ? 0 : l == 2 ? 3 : l == 3 ? 8 : 15;
            constexpr int b1 = l == 1 ? 3 : l == 2 ? 8 : l == 3 ? 15 : 24;
            constexpr int lo = b0 > k0 ? b0 : k0, hi = b1 < k1 ? b1 : k1;
            if constexpr (lo < hi) {
              float acc = q[(NR + 1) + (l - 1) * (NA + 1) + n];
#pragma unroll
              for (int k = lo; k < hi; ++k) acc = __fmaf_rn(w.m.c3b[k] * Sv[n][k - k0], Sv[n][k - k0], acc);
              q[(NR + 1) + (l - 1) * (NA + 1) + n] = acc;
            }
          });
          if constexpr (k0 == 0) {
            if constexpr (S::L4 >= 2) {
              const float s3 = Sv[n][3], s4 = Sv[n][4], s5 = Sv[n][5], s6 = Sv[n][6], s7 = Sv[n][7];
              q[S::OFF4 + n] = w.m.c4b[0] * s3 * s3 * s3 + w.m.c4b[1] * s3 * (s4 * s4 + s5 * s5) +
                               w.m.c4b[2] * s3 * (s6 * s6 + s7 * s7) + w.m.c4b[3] * s6 * (s5 * s5 - s4 * s4) +
                               w.m.c4b[4] * s4 * s5 * s7;
            }
            if constexpr (S::L5 >= 1) {
              const float s0 = Sv[n][0], s12 = Sv[n][1] * Sv[n][1] + Sv[n][2] * Sv[n][2];
              q[S::OFF5 + n] = w.m.c5b[0] * s0 * s0 * s0 * s0 + w.m.c5b[1] * s0 * s0 * s12 + w.m.c5b[2] * s12 * s12;
            }
          }
          if constexpr (TCLR) {
            // park this part of S_n in the thread's shared block (TMEM serves the network)
#pragma unroll
            for (int k4 = 0; k4 < NKC / 4; ++k4)
              sref(n * (NKP / 4) + k0 / 4 + k4) =
                  make_float4(Sv[n][4 * k4], Sv[n][4 * k4 + 1], Sv[n][4 * k4 + 2], Sv[n][4 * k4 + 3]);
          } else {
            // park this part of S_n in TMEM, columns n NK + k0 .. n NK + k1 - 1
            __syncwarp();
#pragma unroll
            for (int k8 = 0; k8 < NKC / 8; ++k8) tmem_st8(tmem_row + n * NK + k0 + 8 * k8, &Sv[n][8 * k8]);
          }
        }
      });
    } else
    static_for<0, NPASS>([&](auto pc) {
      constexpr int n0 = decltype(pc)::value * NCH;
      constexpr int n1 = (n0 + NCH < NA + 1) ? n0 + NCH : NA + 1;
      constexpr int NC = n1 - n0;
      float Sv[NC][NK];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < NK; ++k) Sv[c][k] = 0.f;
      for_pairs(a.nl_a, 0, na, N, i, a.pos4, a.jmask, [&](int, unsigned e, const float4 &pj) {
        const float3 d = pair_vector(pi, pj, shift(e));
        const float r2 = norm2(d);
        if (r2 < rcA2) {
          const int tj = type_of(pj);
          const float rinv = rsqrtf(r2);
          float f[KA + 1];
          cheb_basis<KA>(r2 * rinv, inv_rcA, f);
          const float4 *cc = reinterpret_cast<const float4 *>(cA_s + ((ti * T + tj) * (NA + 1) + n0) * KAP);
          float g[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < KAP / 4; ++k4) {
              const float4 cv = cc[c * (KAP / 4) + k4];
              const float cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (4 * k4 + j <= KA) acc = __fmaf_rn(cw[j], f[4 * k4 + j], acc);
            }
            g[c] = acc;
          }
          const float rl[5] = {1.f, rinv, rinv * rinv, rinv * rinv * rinv, (rinv * rinv) * (rinv * rinv)};
          static_for<0, NK>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const float b = poly_b<k>(d.x, d.y, d.z, r2) * rl[l_of_k(k)];
#pragma unroll
            for (int c = 0; c < NC; ++c) Sv[c][k] = __fmaf_rn(g[c], b, Sv[c][k]);
          });
        }
      });
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int n = n0 + c;
        static_for<0, S::L3>([&](auto lc) {
          constexpr int l = decltype(lc)::value + 1;
          constexpr int k0 = l == 1 ? 0 : l == 2 ? 3 : l == 3 ? 8 : 15;
          constexpr int k1 = l == 1 ? 3 : l == 2 ? 8 : l == 3 ? 15 : 24;
          float acc = 0.f;
#pragma unroll
          for (int k = k0; k < k1; ++k) acc = __fmaf_rn(w.m.c3b[k] * Sv[c][k], Sv[c][k], acc);
          q[(NR + 1) + (l - 1) * (NA + 1) + n] = acc;
        });
        if constexpr (S::L4 >= 2) {
          const float s3 = Sv[c][3], s4 = Sv[c][4], s5 = Sv[c][5], s6 = Sv[c][6], s7 = Sv[c][7];
          q[S::OFF4 + n] = w.m.c4b[0] * s3 * s3 * s3 + w.m.c4b[1] * s3 * (s4 * s4 + s5 * s5) +
                           w.m.c4b[2] * s3 * (s6 * s6 + s7 * s7) + w.m.c4b[3] * s6 * (s5 * s5 - s4 * s4) +
                           w.m.c4b[4] * s4 * s5 * s7;
        }
        if constexpr (S::L5 >= 1) {
          const float s0 = Sv[c][0], s12 = Sv[c][1] * Sv[c][1] + Sv[c][2] * Sv[c][2];
          q[S::OFF5 + n] = w.m.c5b[0] * s0 * s0 * s0 * s0 + w.m.c5b[1] * s0 * s0 * s12 + w.m.c5b[2] * s12 * s12;
        }
        if constexpr (!DESC_ONLY && !TM) {
          // park S_n in this thread's shared block while the network runs
          float4 *dst = reinterpret_cast<float4 *>(S_s + threadIdx.x * SPT + n * NKP);
#pragma unroll
          for (int k4 = 0; k4 < NKP / 4; ++k4) {
            float v4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v4[j] = 4 * k4 + j < NK ? Sv[c][4 * k4 + j] : 0.f;
            dst[k4] = make_float4(v4[0], v4[1], v4[2], v4[3]);
          }
        }
        if constexpr (TM) {
          // park S_n in this thread's TMEM lane, columns n NK .. n NK + NK - 1
          __syncwarp();
#pragma unroll
          for (int k8 = 0; k8 < NK / 8; ++k8) tmem_st8(tmem_row + n * NK + 8 * k8, &Sv[c][8 * k8]);
        }
      }
    });

    if constexpr (DESC_ONLY) {
      if (active) {
        const size_t io = a.perm ? (size_t)a.perm[i] : (size_t)i;
#pragma unroll
        for (int v = 0; v < NDES; ++v) a.q_out[io * NDES + v] = (double)q[v];
      }
    } else {
      if constexpr (TM) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

      // ---- network, Eq. Ui, and dU/dq
      float U = 0.f;
      float dq[NDES];
#pragma unroll
      for (int v = 0; v < NDES; ++v) dq[v] = 0.f;
      if constexpr (PREC == 0) {
        // FP32 on the FMA pipes, weights broadcast from shared memory
  #pragma unroll 1
        for (int mu = 0; mu < S::H; ++mu) {
          const float4 *row = reinterpret_cast<const float4 *>(w0_s + mu * NDP);
          float4 wrow[NDP / 4];  // the row serves both the forward and the backward sum
          float zp[4] = {-b0_s[mu], 0.f, 0.f, 0.f};
  #pragma unroll
          for (int v4 = 0; v4 < NDP / 4; ++v4) {
            const float4 wv = wrow[v4] = row[v4];
            const float wc[4] = {wv.x, wv.y, wv.z, wv.w};
  #pragma unroll
            for (int c = 0; c < 4; ++c)
              if (4 * v4 + c < NDES) zp[c] = __fmaf_rn(wc[c], q[4 * v4 + c], zp[c]);
          }
          const float h = tanhf((zp[0] + zp[1]) + (zp[2] + zp[3]));
          const float w1m = w1_s[mu];
          U = __fmaf_rn(w1m, h, U);
          const float beta = w1m * (1.f - h * h);
  #pragma unroll
          for (int v4 = 0; v4 < NDP / 4; ++v4) {
            const float4 wv = wrow[v4];
            const float wc[4] = {wv.x, wv.y, wv.z, wv.w};
  #pragma unroll
            for (int c = 0; c < 4; ++c)
              if (4 * v4 + c < NDES) dq[4 * v4 + c] = __fmaf_rn(beta, wc[c], dq[4 * v4 + c]);
          }
        }
      } else {
        // BF16 tensor cores (tcgen05), FP32 accumulation in TMEM, one 128-atom tile per block.
        // Every completion wait is bounded; if one runs out (all threads agree through the
        // barrier), the block flags the error, waits once more (again bounded) so that the
        // MMAs in flight finish before the TMEM is read or freed, and skips the rest of the
        // network: its results are then invalid and the host reports NEP_ERR_TIMEOUT.
        static_assert(NK % 8 == 0, "S_nk is moved in groups of 8 TMEM columns");
        constexpr int KC1 = S::KP1 / 8, KC2 = S::KP2 / 8;
        const int r = threadIdx.x;
        // operand row of 8 values: BF16 (round to nearest even) and, split form, the BF16 of
        // the remainder
        auto put8 = [&](unsigned char *hi, unsigned char *lo, int off, const float *x) {
          uint32_t ph[4], pl[4];
#pragma unroll
          for (int h2 = 0; h2 < 4; ++h2) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * h2], x[2 * h2 + 1]);
            ph[h2] = *reinterpret_cast<const uint32_t *>(&b);
            if constexpr (SPLIT)
              pl[h2] = pack_bf16x2(x[2 * h2] - __low2float(b), x[2 * h2 + 1] - __high2float(b));
          }
          *reinterpret_cast<uint4 *>(hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
          if constexpr (SPLIT) *reinterpret_cast<uint4 *>(lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        };
        // one GEMM over K steps of 16: D = A.B^T (+ A_lo.B^T + A.B_lo^T in the split form)
        auto gemm = [&](const unsigned char *A, const unsigned char *Alo, const unsigned char *B,
                        const unsigned char *Blo, int ksteps, int KC, uint32_t idesc) {
          for (int st = 0; st < ksteps; ++st) {
            const uint64_t da = umma_desc(smem_addr(A) + 256 * st, 128, KC * 128);
            const uint64_t db = umma_desc(smem_addr(B) + 256 * st, 128, KC * 128);
            umma_bf16(tc_tmem + S::DCOL, da, db, idesc, st > 0 ? 1u : 0u);
            if constexpr (SPLIT) {
              umma_bf16(tc_tmem + S::DCOL, umma_desc(smem_addr(Alo) + 256 * st, 128, KC * 128), db, idesc, 1u);
              umma_bf16(tc_tmem + S::DCOL, da, umma_desc(smem_addr(Blo) + 256 * st, 128, KC * 128), idesc, 1u);
            }
          }
          umma_commit(&tc_mbar);
        };
        // wait for the commit of phase `parity`; false (block-uniform) if the wait ran out
        auto tc_wait = [&](uint32_t parity) -> bool {
          const bool ok = mbar_wait(&tc_mbar, parity);
          if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(a.tc_err, 1);
            mbar_wait(&tc_mbar, parity);
            return false;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          return true;
        };
        if constexpr (TCLR) {
          // Low-register form: the A operands go to TMEM columns ACOL.. as BF16 pairs (one lane
          // per atom, no shared-memory tile; split form: their lo parts at ALO..), the results
          // to columns 0... GEMM2 reads the GEMM1 tile of W0 MN-major (B = W0).
          constexpr uint32_t ACOL = S::ACOL, ALO = S::ALO;
          // 16 values -> A (and A_lo) columns col .. col + 7
          auto put16 = [&](uint32_t col, const float *x) {
            uint32_t u[8], ul[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const __nv_bfloat162 bh = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
              u[j] = *reinterpret_cast<const uint32_t *>(&bh);
              if constexpr (SPLIT)
                ul[j] = pack_bf16x2(x[2 * j] - __low2float(bh), x[2 * j + 1] - __high2float(bh));
            }
            tmem_st8u(tmem_row + ACOL + col, u);
            if constexpr (SPLIT) tmem_st8u(tmem_row + ALO + col, ul);
          };
          // operands written by every thread -> visible to the MMA issued by thread 0
          auto to_mma = [&]() {
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          };
          // D = A.B over K steps of 16 (+ A_lo.B + A.B_lo in the split form, in the order of
          // the two-CTA form); B step st at byte offset st * bstep, descriptors (lbo, sbo)
          auto gemm_t = [&](const unsigned char *B, const unsigned char *Blo, int ksteps, uint32_t bstep,
                            uint32_t lbo, uint32_t sbo, uint32_t idesc) {
            for (int st = 0; st < ksteps; ++st) {
              const uint64_t db = umma_desc(smem_addr(B) + bstep * st, lbo, sbo);
              umma_bf16_ts(tc_tmem, tc_tmem + ACOL + 8 * st, db, idesc, st > 0 ? 1u : 0u);
              if constexpr (SPLIT) {
                umma_bf16_ts(tc_tmem, tc_tmem + ALO + 8 * st, db, idesc, 1u);
                umma_bf16_ts(tc_tmem, tc_tmem + ACOL + 8 * st, umma_desc(smem_addr(Blo) + bstep * st, lbo, sbo),
                             idesc, 1u);
              }
            }
            umma_commit(&tc_mbar);
          };
#pragma unroll
          for (int c8 = 0; c8 < S::KP1 / 16; ++c8) {  // q row -> A
            float x[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = 16 * c8 + j < NDES ? q[16 * c8 + j] : 0.f;
            put16(8 * c8, x);
          }
          to_mma();
          if (threadIdx.x == 0)  // GEMM1: z = q . W0^T into columns 0 .. NP1 - 1
            gemm_t(tileB1, tileB1lo, S::KP1 / 16, 256, 128, KC1 * 128, umma_idesc_bf16<kAtomBlock, S::NP1>());
          __syncwarp();
          if (tc_wait(0)) {
            // tanh layer from this row of z; beta = w1 (1 - h^2) -> A (16 hidden units per store;
            // the GEMM that read q has completed)
#pragma unroll
            for (int c16 = 0; c16 < S::NP1 / 16; ++c16) {
              float z[16];
              tmem_ld8(tmem_row + 16 * c16, z);
              tmem_ld8(tmem_row + 16 * c16 + 8, z + 8);
              float bt[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int mu = 16 * c16 + j;
                bt[j] = 0.f;
                if (mu < S::H) {
                  const float h = tanhf(z[j] - b0_s[mu]);
                  U = __fmaf_rn(w1_s[mu], h, U);
                  bt[j] = w1_s[mu] * (1.f - h * h);
                }
              }
              put16(8 * c16, bt);
            }
            // every lane has read its z (tcgen05.ld waited) before GEMM2 overwrites the columns
            to_mma();
            // GEMM2: dq = beta . W0 into columns 0 .. NP2 - 1; B = W0 (K = hidden units, N =
            // descriptor components) MN-major from the GEMM1 tile, 16 hidden units (two row
            // groups of KC1 core matrices) per step
            if (threadIdx.x == 0)
              gemm_t(tileB1, tileB1lo, S::KP2 / 16, 2 * KC1 * 128, KC1 * 128, 128,
                     umma_idesc_bf16_bmn<kAtomBlock, S::NP2>());
            __syncwarp();
            if (tc_wait(1)) {
#pragma unroll
              for (int c8 = 0; c8 < S::NP2 / 8; ++c8) {
                float v[8];
                tmem_ld8(tmem_row + 8 * c8, v);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  if (8 * c8 + j < NDES) dq[8 * c8 + j] = v[j];
              }
            }
          }
        } else {
          // q row -> operand tile A (bf16, K-major)
#pragma unroll
          for (int kc = 0; kc < KC1; ++kc) {
            float x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = 8 * kc + j < NDES ? q[8 * kc + j] : 0.f;
            put8(tileA, tileAlo, umma_off(r, 8 * kc, KC1), x);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncthreads();
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (threadIdx.x == 0)  // GEMM1: z = q . W0^T into TMEM columns DCOL ..
            gemm(tileA, tileAlo, tileB1, tileB1lo, S::KP1 / 16, KC1, umma_idesc_bf16<kAtomBlock, S::NP1>());
          __syncwarp();
          if (tc_wait(0)) {
            // tanh layer from this row of z; beta = w1 (1 - h^2) -> operand tile A (reused)
#pragma unroll
            for (int c8 = 0; c8 < S::NP1 / 8; ++c8) {
              float z[8];
              tmem_ld8(tmem_row + S::DCOL + 8 * c8, z);
              float bt[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int mu = 8 * c8 + j;
                bt[j] = 0.f;
                if (mu < S::H) {
                  const float h = tanhf(z[j] - b0_s[mu]);
                  U = __fmaf_rn(w1_s[mu], h, U);
                  bt[j] = w1_s[mu] * (1.f - h * h);
                }
              }
              put8(tileA, tileAlo, umma_off(r, 8 * c8, KC2), bt);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (threadIdx.x == 0)  // GEMM2: dq = beta . W0 into the same TMEM columns
              gemm(tileA, tileAlo, tileB2, tileB2lo, S::KP2 / 16, KC2, umma_idesc_bf16<kAtomBlock, S::NP2>());
            __syncwarp();
            if (tc_wait(1)) {
#pragma unroll
              for (int c8 = 0; c8 < S::NP2 / 8; ++c8) {
                float v[8];
                tmem_ld8(tmem_row + S::DCOL + 8 * c8, v);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  if (8 * c8 + j < NDES) dq[8 * c8 + j] = v[j];
              }
            }
          }
        }
      }
      if constexpr (BATCH) U -= b1_s;
      else U -= w.b1;
      if (active) {
        if (a.energy) a.energy[mem * a.s_out + (a.perm ? a.perm[i] : i)] = (double)U;
        Ublock = (double)U;
      }

      // ---- radial force coefficients e^t_k = sum_n dU/dq_n c^{t_i t}_{nk} and their sum
      for (int t = 0; t < T; ++t) {
        const float4 *c = reinterpret_cast<const float4 *>(cR_s + (ti * T + t) * (NR + 1) * KRP);
        float ev[S::EST > KRP ? S::EST : KRP];
#pragma unroll
        for (int k4 = 0; k4 < KRP / 4; ++k4) {
          float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int n = 0; n <= NR; ++n) {
            const float4 cv = c[n * (KRP / 4) + k4];
            acc[0] = __fmaf_rn(dq[n], cv.x, acc[0]);
            acc[1] = __fmaf_rn(dq[n], cv.y, acc[1]);
            acc[2] = __fmaf_rn(dq[n], cv.z, acc[2]);
            acc[3] = __fmaf_rn(dq[n], cv.w, acc[3]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) ev[4 * k4 + j] = acc[j];
        }
        float tot = 0.f;
#pragma unroll
        for (int k = 0; k <= KR; ++k) tot += ev[k];
        ev[KR + 1] = tot;
#pragma unroll
        for (int k = KR + 2; k < S::EST; ++k) ev[k] = 0.f;
        if (active) {
          float4 *dst = reinterpret_cast<float4 *>(a.e_rad + mem * a.s_erad + ((size_t)i * T + t) * S::EST);
#pragma unroll
          for (int k4 = 0; k4 < S::EST / 4; ++k4)
            dst[k4] = make_float4(ev[4 * k4], ev[4 * k4 + 1], ev[4 * k4 + 2], ev[4 * k4 + 3]);
        }
      }

      // ---- dU/dS_nk from the explicit 3/4/5-body forms, kept in registers for the force loop
      // (low-register form: in this thread's shared block, row n at n NKP)
      float dSr[LOWREG ? 1 : NA + 1][NKP];
#pragma unroll
      for (int n = 0; n <= NA; ++n) {
        float s[NKP];
        float *dS = dSr[LOWREG ? 0 : n];
        if constexpr (!STM) {
#pragma unroll
          for (int k4 = 0; k4 < NKP / 4; ++k4) {
            const float4 v = sref(n * (NKP / 4) + k4);
            s[4 * k4] = v.x, s[4 * k4 + 1] = v.y, s[4 * k4 + 2] = v.z, s[4 * k4 + 3] = v.w;
          }
        } else {
          __syncwarp();
#pragma unroll
          for (int k8 = 0; k8 < NK / 8; ++k8) tmem_ld8(tmem_row + n * NK + 8 * k8, &s[8 * k8]);
        }
#pragma unroll
        for (int k = 0; k < NKP; ++k) {
          if (k < S::KEND3) {
            const float d3 = dq[(NR + 1) + (l_of_k(k) - 1) * (NA + 1) + n];
            dS[k] = 2.f * w.m.c3b[k] * s[k] * d3;
          } else {
            dS[k] = 0.f;
          }
        }
        if constexpr (S::L4 >= 2) {
          const float d4 = dq[S::OFF4 + n];
          const float *C = w.m.c4b;
          dS[3] += d4 * (3.f * C[0] * s[3] * s[3] + C[1] * (s[4] * s[4] + s[5] * s[5]) + C[2] * (s[6] * s[6] + s[7] * s[7]));
          dS[4] += d4 * (2.f * C[1] * s[3] * s[4] - 2.f * C[3] * s[6] * s[4] + C[4] * s[5] * s[7]);
          dS[5] += d4 * (2.f * C[1] * s[3] * s[5] + 2.f * C[3] * s[6] * s[5] + C[4] * s[4] * s[7]);
          dS[6] += d4 * (2.f * C[2] * s[3] * s[6] + C[3] * (s[5] * s[5] - s[4] * s[4]));
          dS[7] += d4 * (2.f * C[2] * s[3] * s[7] + C[4] * s[4] * s[5]);
        }
        if constexpr (S::L5 >= 1) {
          const float d5 = dq[S::OFF5 + n];
          const float *C = w.m.c5b;
          const float s12 = s[1] * s[1] + s[2] * s[2];
          dS[0] += d5 * (4.f * C[0] * s[0] * s[0] * s[0] + 2.f * C[1] * s[0] * s12);
          const float common = 2.f * C[1] * s[0] * s[0] + 4.f * C[2] * s12;
          dS[1] += d5 * common * s[1];
          dS[2] += d5 * common * s[2];
        }
        if constexpr (LOWREG) {
#pragma unroll
          for (int k4 = 0; k4 < NKP / 4; ++k4)
            sref(n * (NKP / 4) + k4) = make_float4(dS[4 * k4], dS[4 * k4 + 1], dS[4 * k4 + 2], dS[4 * k4 + 3]);
        }
      }

      // ---- angular partial forces dU_i/dr_ij (angular terms of Eq. partial_force)
      for_pairs(a.nl_a, 0, na, N, i, a.pos4, a.jmask, [&](int m, unsigned e, const float4 &pj) {
        const float3 d = pair_vector(pi, pj, shift(e));
        const float r2 = norm2(d);
        if (r2 < rcA2) {
          const int tj = type_of(pj);
          const float rinv = rsqrtf(r2);
          float f[KA + 1], fp[KA + 1];
          cheb_basis_d<KA>(r2 * rinv, inv_rcA, f, fp);
          const float4 *c = reinterpret_cast<const float4 *>(cA_s + (ti * T + tj) * (NA + 1) * KAP);
          float g[NA + 1], gp[NA + 1];
#pragma unroll
          for (int n = 0; n <= NA; ++n) {
            float acc = 0.f, accp = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < KAP / 4; ++k4) {
              const float4 cv = c[n * (KAP / 4) + k4];
              const float cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (4 * k4 + j <= KA) {
                  acc = __fmaf_rn(cw[j], f[4 * k4 + j], acc);
                  accp = __fmaf_rn(cw[j], fp[4 * k4 + j], accp);
                }
            }
            g[n] = acc;
            gp[n] = accp;
          }
          // G = sum_k a_k r^-l grad b_k (tangential part used), Y = sum_k c_k r^-l b_k
          const float rl[5] = {1.f, rinv, rinv * rinv, rinv * rinv * rinv, (rinv * rinv) * (rinv * rinv)};
          float gx = 0.f, gy = 0.f, gz = 0.f, yy = 0.f;
          static_for<0, NKP / 4>([&](auto kq) {
            constexpr int k0 = 4 * decltype(kq)::value;
            float ak[4] = {0.f, 0.f, 0.f, 0.f}, ck[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int n = 0; n <= NA; ++n) {
              float dv[4];
              if constexpr (LOWREG) {
                const float4 v = sref(n * (NKP / 4) + k0 / 4);
                dv[0] = v.x, dv[1] = v.y, dv[2] = v.z, dv[3] = v.w;
              } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) dv[j] = k0 + j < NK ? dSr[n][k0 + j] : 0.f;
              }
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (k0 + j < NK) {
                  ak[j] = __fmaf_rn(dv[j], g[n], ak[j]);
                  ck[j] = __fmaf_rn(dv[j], gp[n], ck[j]);
                }
            }
            static_for<0, 4>([&](auto jc) {
              constexpr int j = decltype(jc)::value, k = k0 + j;
              if constexpr (k < NK) {
                const float akr = ak[j] * rl[l_of_k(k)], ckr = ck[j] * rl[l_of_k(k)];
                const float3 gb = poly_grad<k>(d.x, d.y, d.z, r2);
                gx = __fmaf_rn(akr, gb.x, gx);
                gy = __fmaf_rn(akr, gb.y, gy);
                gz = __fmaf_rn(akr, gb.z, gz);
                yy = __fmaf_rn(ckr, poly_b<k>(d.x, d.y, d.z, r2), yy);
              }
            });
          });
          const float ux = d.x * rinv, uy = d.y * rinv, uz = d.z * rinv;
          const float gu = gx * ux + gy * uy + gz * uz;
          const float px = (gx - gu * ux) + yy * ux;
          const float py = (gy - gu * uy) + yy * uy;
          const float pz = (gz - gu * uz) + yy * uz;
          a.p_ang[mem * a.s_pang + (size_t)m * N + i] = make_float4(px, py, pz, 0.f);
        }
      });
    }
  }
  if constexpr (!DESC_ONLY) {
    // deterministic block sum of U (fixed shuffle tree, then fixed warp order)
    __shared__ double red[AB / 32];
    double v = Ublock;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int wv = 0; wv < AB / 32; ++wv) s += red[wv];
      a.partial_atom[(size_t)mem * gridDim.x + blockIdx.x] = s;
    }
  }
  if constexpr (TM) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc_tmem), "r"(TCOLS));
    }
  }
}

// Epilogue of the gather kernels for atom i: outputs in the caller's order, the squared force
// error of Eq. loss, the second velocity-Verlet half-kick with the kinetic energy, and the
// heat current J_i = W_i . v_i (Eq. Ji); part[] collects the block sums.
__device__ __forceinline__ void gather_epilogue(const AtomArgs &a, int i, const float4 &pi, int ti, int mem,
                                                float fx, float fy, float fz, const float *w, double *part) {
  const double Fx = fx, Fy = fy, Fz = fz;
  const size_t io = mem * a.s_out + (a.perm ? (size_t)a.perm[i] : (size_t)i);
  if (a.force) {
    a.force[3 * io] = Fx;
    a.force[3 * io + 1] = Fy;
    a.force[3 * io + 2] = Fz;
  }
  if (a.virial) {
#pragma unroll
    for (int c = 0; c < 9; ++c) a.virial[9 * io + c] = (double)w[c];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) part[2 + c] = (double)w[c];
  // velocity of the heat current: after the kick below (MD), or given by the caller
  double vh[3] = {0.0, 0.0, 0.0};
  if (a.vel_in) {
    const double *vi = a.vel_in + 3 * (a.perm ? (size_t)a.perm[i] : (size_t)i);
    vh[0] = vi[0]; vh[1] = vi[1]; vh[2] = vi[2];
  }
  if (a.f_tar) {  // squared force error against target forces (the force term of Eq. loss)
    const double *ft = a.f_tar + 3 * (a.perm ? (size_t)a.perm[i] : (size_t)i);
    const double ex = Fx - ft[0], ey = Fy - ft[1], ez = Fz - ft[2];
    part[11] = ex * ex + ey * ey + ez * ez;
  }
  bool kick = a.md_kick && !(a.fire && a.fire->converged);
  double hdt = a.fire ? 0.5 * a.fire->dt : a.half_dt;
  if (a.slots) {  // batched engine: the structure's own phase and time step
    const EngineSlot &sl = a.slots[struct_of(pi)];
    kick = sl.phase == 1 && !(sl.kind == kJobFire && sl.fire.converged);
    hdt = 0.5 * (sl.kind == kJobFire ? sl.fire.dt : sl.dt);
  }
  if (kick) {  // second half-kick of velocity Verlet, kinetic energy
    double *v = a.vel + 3 * (size_t)i;
    const double s = hdt * a.inv_mass_kappa[ti];
    const double vx = v[0] + s * Fx, vy = v[1] + s * Fy, vz = v[2] + s * Fz;
    v[0] = vx; v[1] = vy; v[2] = vz;
    part[1] = a.mass_kappa_half[ti] * (vx * vx + vy * vy + vz * vz);
    vh[0] = vx; vh[1] = vy; vh[2] = vz;
  } else if (a.md_kick || a.slots) {  // converged FIRE or no step: velocities unchanged
    const double *v = a.vel + 3 * (size_t)i;
    part[1] = a.mass_kappa_half[ti] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    vh[0] = v[0]; vh[1] = v[1]; vh[2] = v[2];
  }
  // J_i = W_i . v_i, W_i[a][b] in the order xx, yy, zz, xy, xz, yz, yx, zx, zy (Eq. Ji)
  const double Jx = (double)w[0] * vh[0] + (double)w[3] * vh[1] + (double)w[4] * vh[2];
  const double Jy = (double)w[6] * vh[0] + (double)w[1] * vh[1] + (double)w[5] * vh[2];
  const double Jz = (double)w[7] * vh[0] + (double)w[8] * vh[1] + (double)w[2] * vh[2];
  part[12] = Jx;
  part[13] = Jy;
  part[14] = Jz;
  if (a.heat) {
    a.heat[3 * io] = Jx;
    a.heat[3 * io + 1] = Jy;
    a.heat[3 * io + 2] = Jz;
  }
}

// Deterministic block sums of (KE, W[9], force error, J[3]) over a block of GB threads.
template <int GB>
__device__ __forceinline__ void gather_block_sums(const AtomArgs &a, int mem, const double *part) {
  __shared__ double red[GB / 32][kReduceSlots];
#pragma unroll
  for (int s = 1; s < kReduceSlots; ++s) {
    double v = part[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][s] = v;
  }
  __syncthreads();
  if (threadIdx.x < kReduceSlots && threadIdx.x >= 1) {
    double s = 0.0;
    for (int wv = 0; wv < GB / 32; ++wv) s += red[wv][threadIdx.x];
    a.partial_gather[((size_t)mem * gridDim.x + blockIdx.x) * kReduceSlots + threadIdx.x] = s;
  }
}

// ------------------------------------------------------------------------ gather kernel
// For one structure the gather is held to 64 registers for N_bas^R <= 8 (1024 threads per SM:
// 8 CTAs of 128 instead of 7 hide more of the neighbour gathers' latency; 8,000,000 Si atoms:
// 3.17 against 3.52 ms) and to 72 above (7 CTAs); the batched form keeps the compiler's choice.
template <class S, bool BATCH = false, int GB = kGatherBlock>
__global__ void __launch_bounds__(GB, BATCH ? 1 : (S::KR <= 8 ? 1024 : 896) / GB)
    gather_kernel(const AtomArgs a) {
  constexpr int KR = S::KR, EST = S::EST;
  extern __shared__ float4 smem4[];
  float4 *dtab_s = smem4;
  const int mem = BATCH ? (int)blockIdx.y : 0;
  if constexpr (!BATCH) {
    for (int v = threadIdx.x; v < a.ncode; v += blockDim.x) dtab_s[v] = a.dtab[v];
    __syncthreads();
  }
  const float *e_rad = a.e_rad + mem * a.s_erad;
  const float4 *p_ang = a.p_ang + mem * a.s_pang;
  const int N = a.N, T = a.T;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part[kReduceSlots];
#pragma unroll
  for (int s = 0; s < kReduceSlots; ++s) part[s] = 0.0;
  // (serving engine) atoms of a finished job frozen in the batch are skipped
  if (i < N && !(BATCH && a.slots && a.slots[struct_of(a.pos4[i])].phase == 2)) {
    const float4 pi = a.pos4[i];
    const int ti = type_of(pi);
    const float4 *dtab_b = BATCH ? a.dtab + (size_t)struct_of(pi) * a.ncode : dtab_s;
    auto shift = [&](unsigned e) -> float4 {
      if constexpr (BATCH) return __ldg(dtab_b + (e >> a.jbits));
      else return dtab_s[e >> a.jbits];
    };
    const float inv_rcR = 1.f / a.rcR;
    const float rcR2 = a.rcR * a.rcR, rcA2 = a.rcA * a.rcA;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float w[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) w[c] = 0.f;
    // ---- radial part (Algorithm 2): s_i from own e^{t_j}, s_j from neighbour's e^{t_i}
    int base = 0;
    for (int t = 0; t < T; ++t) {
      const int cnt = a.nn_r[t * N + i];
      float eo[EST];
      const float4 *src = reinterpret_cast<const float4 *>(e_rad + ((size_t)i * T + t) * EST);
#pragma unroll
      for (int k4 = 0; k4 < EST / 4; ++k4) {
        const float4 v = src[k4];
        eo[4 * k4] = v.x; eo[4 * k4 + 1] = v.y; eo[4 * k4 + 2] = v.z; eo[4 * k4 + 3] = v.w;
      }
      for_pairs_batch<2, true, 1>(a.nl_r, base, cnt, N, i, a.pos4, a.jmask, [&](int, unsigned e, const float4 &pj) {
        const int j = e & a.jmask;
        const float3 d = pair_vector(pi, pj, shift(e));
        const float r2 = norm2(d);
        if (r2 < rcR2) {
          const float rinv = rsqrtf(r2);
          const float r = r2 * rinv;
          float ej[EST];
          const float4 *srcj = reinterpret_cast<const float4 *>(e_rad + ((size_t)j * T + ti) * EST);
#pragma unroll
          for (int k4 = 0; k4 < EST / 4; ++k4) {
            const float4 v = __ldg(srcj + k4);
            ej[4 * k4] = v.x; ej[4 * k4 + 1] = v.y; ej[4 * k4 + 2] = v.z; ej[4 * k4 + 3] = v.w;
          }
          // sum_k e_k f_k'(r) = (x' fc/2) sum_k e_k T_k'(x) + (fc'/2) (sum_k e_k T_k(x) + sum_k e_k)
          const float u = r * inv_rcR;
          float sn, cs;
          __sincosf(3.14159265358979f * u, &sn, &cs);
          const float hfc = 0.25f * (1.f + cs);
          const float hfcp = -0.25f * 3.14159265358979f * inv_rcR * sn;
          const float t1 = u - 1.f;
          const float x = 2.f * t1 * t1 - 1.f;
          const float xp = 4.f * t1 * inv_rcR;
          const float x2 = 2.f * x;
          float tkm1 = 1.f, tk = x, dkm1 = 0.f, dk = 1.f;
          float oT = eo[0], oD = 0.f, jT = ej[0], jD = 0.f;
          if (KR >= 1) {
            oT = __fmaf_rn(eo[1], x, oT);
            jT = __fmaf_rn(ej[1], x, jT);
            oD = eo[1];
            jD = ej[1];
          }
#pragma unroll
          for (int k = 2; k <= KR; ++k) {
            const float tn = __fmaf_rn(x2, tk, -tkm1);
            const float dn = __fmaf_rn(x2, dk, __fmaf_rn(2.f, tk, -dkm1));
            tkm1 = tk; tk = tn; dkm1 = dk; dk = dn;
            oT = __fmaf_rn(eo[k], tn, oT);
            jT = __fmaf_rn(ej[k], tn, jT);
            oD = __fmaf_rn(eo[k], dn, oD);
            jD = __fmaf_rn(ej[k], dn, jD);
          }
          const float a1 = xp * hfc;
          const float si = __fmaf_rn(a1, oD, hfcp * (oT + eo[KR + 1]));
          const float sj = __fmaf_rn(a1, jD, hfcp * (jT + ej[KR + 1]));
          const float fs = (si + sj) * rinv;
          fx = __fmaf_rn(fs, d.x, fx);
          fy = __fmaf_rn(fs, d.y, fy);
          fz = __fmaf_rn(fs, d.z, fz);
          // W_i += r_ij (x) dU_j/dr_ji with dU_j/dr_ji = -s_j d / r
          const float ws = -sj * rinv;
          const float px = ws * d.x, py = ws * d.y, pz = ws * d.z;
          w[0] = __fmaf_rn(d.x, px, w[0]);
          w[1] = __fmaf_rn(d.y, py, w[1]);
          w[2] = __fmaf_rn(d.z, pz, w[2]);
          w[3] = __fmaf_rn(d.x, py, w[3]);
          w[4] = __fmaf_rn(d.x, pz, w[4]);
          w[5] = __fmaf_rn(d.y, pz, w[5]);
          w[6] = __fmaf_rn(d.y, px, w[6]);
          w[7] = __fmaf_rn(d.z, px, w[7]);
          w[8] = __fmaf_rn(d.z, py, w[8]);
        }
      });
      base += cnt;
    }
    // ---- angular part (Algorithm 4): F_i += P_ij - P_ji, W_i += r_ij (x) P_ji
    // Software-pipelined: list entry and reverse slot two entries ahead, the neighbour's
    // position and both partial forces one entry ahead (every reverse slot is a valid slot,
    // and a slot's partial force is used only when the pair is inside the cutoff, which is
    // exactly when the per-atom kernel wrote it).
    const int na = a.nn_a[i];
    if (na > 0) {
      const unsigned *col = a.nl_a + i;
      const int *rcol = a.rev_a + i;
      unsigned e0 = __ldcs(col), e1 = na > 1 ? __ldcs(col + N) : 0u;
      int r1 = na > 1 ? __ldcs(rcol + N) : 0;
      float4 p0 = __ldg(a.pos4 + (e0 & a.jmask));
      float4 pij0 = __ldcs(p_ang + i), pji0 = __ldg(p_ang + __ldcs(rcol));
      for (int m = 0; m < na; ++m) {
        const unsigned e = e0;
        const float4 pj = p0, pij = pij0, pji = pji0;
        if (m + 1 < na) {
          p0 = __ldg(a.pos4 + (e1 & a.jmask));
          pij0 = __ldcs(p_ang + (size_t)(m + 1) * N + i);
          pji0 = __ldg(p_ang + r1);
        }
        e0 = e1;
        if (m + 2 < na) {
          e1 = __ldcs(col + (size_t)(m + 2) * N);
          r1 = __ldcs(rcol + (size_t)(m + 2) * N);
        }
        const float3 d = pair_vector(pi, pj, shift(e));
        const float r2 = norm2(d);
        if (r2 < rcA2) {
          fx += pij.x - pji.x;
          fy += pij.y - pji.y;
          fz += pij.z - pji.z;
          w[0] = __fmaf_rn(d.x, pji.x, w[0]);
          w[1] = __fmaf_rn(d.y, pji.y, w[1]);
          w[2] = __fmaf_rn(d.z, pji.z, w[2]);
          w[3] = __fmaf_rn(d.x, pji.y, w[3]);
          w[4] = __fmaf_rn(d.x, pji.z, w[4]);
          w[5] = __fmaf_rn(d.y, pji.z, w[5]);
          w[6] = __fmaf_rn(d.y, pji.x, w[6]);
          w[7] = __fmaf_rn(d.z, pji.x, w[7]);
          w[8] = __fmaf_rn(d.z, pji.y, w[8]);
        }
      }
    }
    gather_epilogue(a, i, pi, ti, mem, fx, fy, fz, w, part);
  }
  gather_block_sums<GB>(a, mem, part);
}

// ------------------------------------------------------------------------ launchers
// Raise a kernel's dynamic shared memory limit once, to a bound that covers every launch
// (any type count up to kMaxTypes, the largest shift table). The attribute is per function
// and process-wide: setting it per launch to that launch's size would race between threads
// launching the same kernel with different sizes.
template <class K>
cudaError_t smem_limit_once(K kern, size_t bound) {
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> done;
  std::lock_guard<std::mutex> lk(mu);
  const void *key = reinterpret_cast<const void *>(kern);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bound) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bound);
  if (e == cudaSuccess) done[key] = bound;
  return e;
}

template <class S>
size_t atom_smem_bytes(int T, int ncode, int prec, int ab = kAtomBlock, bool tclr = false) {
  // the last region: BF16 operand tiles (tensor-core network; tclr: the per-thread S_nk blocks
  // and the B tiles), nothing (S_nk in TMEM) or the per-thread S_nk blocks
  const bool tm = ab == 128 && S::NK % 8 == 0;
  const size_t last = tclr        ? sizeof(float) * (size_t)S::SPTC * ab + 128 + (prec == 2 ? 2 : 1) * (size_t)S::TILE_B
                      : prec == 1 ? (size_t)S::TILE_A + 2 * S::TILE_B + 128
                      : prec == 2 ? 2 * (size_t)S::TILE_A + 4 * S::TILE_B + 128
                      : tm        ? 0
                                  : sizeof(float) * S::SPT * ab;
  return sizeof(float4) * ncode + sizeof(float) * (size_t)S::off_S(prec, T) + last;
}

// A block that holds TMEM takes 256 of the SM's 512 columns; a third such block on one SM
// would wait in tcgen05.alloc until one of the others ends. When the registers alone would
// admit three blocks, ask for more than a third of the SM's 228 KB of shared memory.
constexpr size_t kTmemBlockSmem = 80 * 1024;
template <class K>
size_t tmem_block_smem(K kern, int block, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void *, int> regs;  // registers per thread of each kernel
  int nr = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    const void *key = reinterpret_cast<const void *>(kern);
    auto it = regs.find(key);
    if (it != regs.end()) {
      nr = it->second;
    } else {
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return smem < kTmemBlockSmem ? kTmemBlockSmem : smem;
      nr = regs[key] = fa.numRegs;
    }
  }
  const int regs_warp = (nr * 32 + 255) / 256 * 256;
  const int by_regs = 65536 / (regs_warp * ((block + 31) / 32));
  return by_regs > 2 && smem < kTmemBlockSmem ? kTmemBlockSmem : smem;
}

template <class S>
cudaError_t launch_atom(const AtomArgs &a, const ModelF &mf, const float *w0, const float *b0, const float *w1,
                        float b1, int descriptor_only, cudaStream_t st) {
  if (a.N <= 0) return cudaSuccess;
  AnnConst<S> w;  // host staging; copied into the launch by value
  for (int v = 0; v < S::H * S::NDES; ++v) w.w0[v] = w0[v];
  for (int v = 0; v < S::H; ++v) {
    w.b0[v] = b0[v];
    w.w1[v] = w1[v];
  }
  w.b1 = b1;
  w.m = mf;
  const int blocks = (a.N + kAtomBlock - 1) / kAtomBlock;
  const bool tm = !descriptor_only && kAtomBlock == 128 && S::NK % 8 == 0;
  size_t smem = atom_smem_bytes<S>(a.T, a.ncode, descriptor_only ? 0 : a.precision);
  size_t bound = atom_smem_bytes<S>(kMaxTypes, 1 << 9, descriptor_only ? 0 : a.precision);
  if (tm && bound < kTmemBlockSmem) bound = kTmemBlockSmem;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit_once(kern, bound);
    if (e != cudaSuccess) return e;
    if (tm) smem = tmem_block_smem(kern, kAtomBlock, smem);
    kern<<<blocks, kAtomBlock, smem, st>>>(a, w);
    return cudaGetLastError();
  };
  if (descriptor_only) return go(atom_kernel<S, true, 0>);
  // low-register form of the tensor-core networks (BF16, split BF16)
  auto go_tclr = [&](auto kern, int prec) -> cudaError_t {
    cudaError_t e = smem_limit_once(kern, atom_smem_bytes<S>(kMaxTypes, 1 << 9, prec, 128, true));
    if (e != cudaSuccess) return e;
    kern<<<blocks, kAtomBlock, atom_smem_bytes<S>(a.T, a.ncode, prec, 128, true), st>>>(a, w);
    return cudaGetLastError();
  };
  if constexpr (S::TCLR_OK)
    if (a.precision == 1 && a.atom_occ == 3) return go_tclr(atom_kernel<S, false, 1, false, 128, 3>, 1);
  if constexpr (S::TCLR2_OK)
    if (a.precision == 2 && a.atom_occ == 3) return go_tclr(atom_kernel<S, false, 2, false, 128, 3>, 2);
  if (a.precision == 1) return go(atom_kernel<S, false, 1>);
  if (a.precision == 2) return go(atom_kernel<S, false, 2>);
  if constexpr (S::NS <= 128 && S::NK % 8 == 0) {
    if (a.atom_occ == 3) {  // low-register form: the per-thread dU/dS_nk blocks, no TMEM-driven cap
      auto kern = atom_kernel<S, false, 0, false, 128, 3>;
      const size_t extra = sizeof(float) * (size_t)S::SPT * kAtomBlock;
      cudaError_t e = smem_limit_once(kern, atom_smem_bytes<S>(kMaxTypes, 1 << 9, 0) + extra);
      if (e != cudaSuccess) return e;
      kern<<<blocks, kAtomBlock, atom_smem_bytes<S>(a.T, a.ncode, 0) + extra, st>>>(a, w);
      return cudaGetLastError();
    }
  }
  return go(atom_kernel<S, false, 0>);
}

template <class S>
cudaError_t launch_gather(const AtomArgs &a, cudaStream_t st) {
  if (a.N <= 0) return cudaSuccess;
  const int blocks = (a.N + kGatherBlock - 1) / kGatherBlock;
  gather_kernel<S><<<blocks, kGatherBlock, sizeof(float4) * a.ncode, st>>>(a);
  return cudaGetLastError();
}

// Batched launches (grid.y = population members); instantiated in the nep_batch_*.cu units.
template <class S>
cudaError_t launch_atom_batch(const AtomArgs &a, const ModelF &mf, const float *w0, const float *b0,
                              const float *w1, float b1, int members, int block, cudaStream_t st);
template <class S>
cudaError_t launch_gather_batch(const AtomArgs &a, int members, int block, cudaStream_t st);

#ifdef NEP_BATCH_KERNELS
template <class S>
cudaError_t launch_atom_batch(const AtomArgs &a, const ModelF &mf, const float *w0, const float *b0,
                              const float *w1, float b1, int members, int block, cudaStream_t st) {
  if (a.N <= 0 || members <= 0) return cudaSuccess;
  if (block != 64 && block != 128) return cudaErrorInvalidValue;
  if (a.precision >= 1 && block != 128) return cudaErrorInvalidValue;
  AnnConst<S> w;
  for (int v = 0; v < S::H * S::NDES; ++v) w.w0[v] = w0 ? w0[v] : 0.f;
  for (int v = 0; v < S::H; ++v) {
    w.b0[v] = b0 ? b0[v] : 0.f;
    w.w1[v] = w1 ? w1[v] : 0.f;
  }
  w.b1 = b1;
  w.m = mf;
  const dim3 grid((a.N + block - 1) / block, members);
  const bool tm = block == 128 && S::NK % 8 == 0;
  size_t smem = atom_smem_bytes<S>(a.T, 0, a.precision, block);
  size_t bound = atom_smem_bytes<S>(kMaxTypes, 0, a.precision, block);
  if (tm && bound < kTmemBlockSmem) bound = kTmemBlockSmem;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit_once(kern, bound);
    if (e != cudaSuccess) return e;
    if (tm) smem = tmem_block_smem(kern, block, smem);
    kern<<<grid, block, smem, st>>>(a, w);
    return cudaGetLastError();
  };
  // the low-register tensor-core forms
  auto go_tclr = [&](auto kern, int prec) -> cudaError_t {
    cudaError_t e = smem_limit_once(kern, atom_smem_bytes<S>(kMaxTypes, 0, prec, 128, true));
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, atom_smem_bytes<S>(a.T, 0, prec, 128, true), st>>>(a, w);
    return cudaGetLastError();
  };
  if constexpr (S::TCLR_OK)
    if (a.precision == 1 && a.atom_occ == 3) return go_tclr(atom_kernel<S, false, 1, true, 128, 3>, 1);
  if constexpr (S::TCLR2_OK)
    if (a.precision == 2 && a.atom_occ == 3) return go_tclr(atom_kernel<S, false, 2, true, 128, 3>, 2);
  if (a.precision == 1) return go(atom_kernel<S, false, 1, true, 128>);
  if (a.precision == 2) return go(atom_kernel<S, false, 2, true, 128>);
  if (block == 64) return go(atom_kernel<S, false, 0, true, 64>);
  if constexpr (S::NS <= 128 && S::NK % 8 == 0) {
    if (a.atom_occ == 3) {  // the low-register form, as in the single-structure launch
      auto kern = atom_kernel<S, false, 0, true, 128, 3>;
      const size_t extra = sizeof(float) * (size_t)S::SPT * 128;
      cudaError_t e = smem_limit_once(kern, atom_smem_bytes<S>(kMaxTypes, 0, 0, 128) + extra);
      if (e != cudaSuccess) return e;
      kern<<<grid, 128, atom_smem_bytes<S>(a.T, 0, 0, 128) + extra, st>>>(a, w);
      return cudaGetLastError();
    }
  }
  return go(atom_kernel<S, false, 0, true, 128>);
}

template <class S>
cudaError_t launch_gather_batch(const AtomArgs &a, int members, int block, cudaStream_t st) {
  if (a.N <= 0 || members <= 0) return cudaSuccess;
  const dim3 grid((a.N + block - 1) / block, members);
  if (block == 64) gather_kernel<S, true, 64><<<grid, 64, 0, st>>>(a);
  else if (block == 128) gather_kernel<S, true, 128><<<grid, 128, 0, st>>>(a);
  else if (block == 256) gather_kernel<S, true, 256><<<grid, 256, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class S>
void attach_batch(ShapeOps &o) {
  o.atom_batch = &launch_atom_batch<S>;
  o.gather_batch = &launch_gather_batch<S>;
}
#else
template <class S>
void attach_batch(ShapeOps &o);  // explicitly instantiated in the batch translation unit
#endif

template <class S> int atom_blocks(int N) { return (N + kAtomBlock - 1) / kAtomBlock; }
template <class S> int gather_blocks(int N) { return (N + kGatherBlock - 1) / kGatherBlock; }

template <class S>
ShapeOps make_ops() {
  ShapeOps o;
  o.nR = S::NR; o.KR = S::KR; o.nA = S::NA; o.KA = S::KA; o.H = S::H;
  o.L3 = S::L3; o.L4 = S::L4; o.L5 = S::L5; o.n_des = S::NDES;
  o.kp1 = S::KP1; o.np1 = S::NP1;
  o.atom = &launch_atom<S>;
  o.gather = &launch_gather<S>;
  o.atom_blocks = &atom_blocks<S>;
  o.gather_blocks = &gather_blocks<S>;
  o.lowreg = (S::NS <= 128 && S::NK % 8 == 0) ? 1 : 0;
  attach_batch<S>(o);
  return o;
}

}  // namespace nep
