/*
 * FP64 CPU oracle for the NEP3 per-step evaluation of arXiv:2205.10046:
 * site energies, forces and per-atom virials (Sec. II), plus the velocity-Verlet
 * NVE step that surrounds it in molecular dynamics.
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the CPU
 * baseline leg of bench.py are the only users. It shares no code, header, table or
 * constant with the CUDA path, and never includes anything from it.
 *
 * It is deliberately plain and slow. Every quantity is FP64 and follows the paper's
 * definitions in the paper's order:
 *   neighbours    every (j, periodic image n) with |r_j + n.H - r_i| < r_c, found by
 *                 brute force over all atoms j and all images that can lie inside the
 *                 cutoff (n is skipped only when one axis alone already puts the image
 *                 beyond r_c);
 *   radial        Eq. qin with g_n of Eq. g_n, f_k of Eq. f_n and the cosine cutoff f_c
 *                 (Sec. II B);
 *   angular       the sums S_{n,k} of Eq. S_nk (Sec. II D) with the 24 polynomials b_k
 *                 exactly as printed, divided by r^l (l = 1, 2, 3, 4 for k in 0-2, 3-7,
 *                 8-14, 15-23), i.e. b_k evaluated on the unit vector; q_nl from the
 *                 printed 3-body coefficients, q_n222 from the printed 4-body ones and
 *                 q_n1111 from the printed 5-body ones;
 *   network       Eq. Ui (single tanh hidden layer);
 *   partial force dU_i/dr_ij of Eq. partial_force, obtained by forward-mode dual numbers
 *                 through all of the above, seeded on one neighbour pair at a time, so no
 *                 derivative is written by hand;
 *   force         Eqs. F_ij and F_i;  virial  Eq. virial (9 components per atom);
 *   dynamics      velocity Verlet; positions wrapped into the cell after every drift and
 *                 the neighbours rebuilt by brute force at every step.
 *
 * Readings taken where the text is garbled or silent: r_ij^n in Eq. S_nk is read as
 * r_ij^l; the angular part uses r_c^A in both the cutoff function and the Chebyshev
 * argument; pairs with r >= r_c are excluded; the descriptor vector is ordered as
 * [radial n = 0..n_R | l = 1 block | l = 2 | l = 3 | l = 4 | 4-body | 5-body], each
 * angular block holding n = 0..n_A; b^(1) is subtracted once per site energy.
 */
#include <cmath>
#include <cstring>
#include <vector>
#include <array>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
  int n_types;
  int n_max_r, n_max_a;   /* n_max^R, n_max^A */
  int basis_r, basis_a;   /* N_bas^R, N_bas^A */
  int l_max_3b, l_max_4b, l_max_5b;
  int n_neuron;
  double rc_r, rc_a;
  const double *c_r;      /* [T][T][n_R+1][K_R+1], ordered type pair (t_i, t_j) */
  const double *c_a;      /* [T][T][n_A+1][K_A+1] */
  const double *w0;       /* [N_neu][N_des] */
  const double *b0;       /* [N_neu] */
  const double *w1;       /* [N_neu] */
  double b1;
} oracle_model;
}

namespace {

const double PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- dual numbers */
/* Value plus gradient with respect to the three components of one pair vector. */
struct Dual {
  double v;
  double g[3];
  Dual() : v(0) { g[0] = g[1] = g[2] = 0; }
  Dual(double x) : v(x) { g[0] = g[1] = g[2] = 0; }
};
inline Dual operator+(const Dual &a, const Dual &b) {
  Dual r(a.v + b.v);
  for (int c = 0; c < 3; ++c) r.g[c] = a.g[c] + b.g[c];
  return r;
}
inline Dual operator-(const Dual &a, const Dual &b) {
  Dual r(a.v - b.v);
  for (int c = 0; c < 3; ++c) r.g[c] = a.g[c] - b.g[c];
  return r;
}
inline Dual operator-(const Dual &a) {
  Dual r(-a.v);
  for (int c = 0; c < 3; ++c) r.g[c] = -a.g[c];
  return r;
}
inline Dual operator*(const Dual &a, const Dual &b) {
  Dual r(a.v * b.v);
  for (int c = 0; c < 3; ++c) r.g[c] = a.g[c] * b.v + a.v * b.g[c];
  return r;
}
inline Dual operator/(const Dual &a, const Dual &b) {
  Dual r(a.v / b.v);
  for (int c = 0; c < 3; ++c) r.g[c] = (a.g[c] * b.v - a.v * b.g[c]) / (b.v * b.v);
  return r;
}
inline Dual &operator+=(Dual &a, const Dual &b) { a = a + b; return a; }
inline Dual sqrt(const Dual &a) {
  Dual r(std::sqrt(a.v));
  for (int c = 0; c < 3; ++c) r.g[c] = a.g[c] / (2.0 * r.v);
  return r;
}
inline Dual cos(const Dual &a) {
  Dual r(std::cos(a.v));
  double s = -std::sin(a.v);
  for (int c = 0; c < 3; ++c) r.g[c] = s * a.g[c];
  return r;
}
inline Dual tanh(const Dual &a) {
  Dual r(std::tanh(a.v));
  double s = 1.0 - r.v * r.v;
  for (int c = 0; c < 3; ++c) r.g[c] = s * a.g[c];
  return r;
}
inline double value(double x) { return x; }
inline double value(const Dual &x) { return x.v; }
using std::sqrt;
using std::cos;
using std::tanh;

/* ---------------------------------------------------------------- model */
struct Model {
  int T, nR, nA, KR, KA, l3, l4, l5, H;
  double rcR, rcA;
  const double *cR, *cA, *w0, *b0, *w1;
  double b1;
  int n_blocks() const { return l3 + (l4 >= 2 ? 1 : 0) + (l5 >= 1 ? 1 : 0); }
  int ndes() const { return (nR + 1) + (nA + 1) * n_blocks(); }
  double c_radial(int ti, int tj, int n, int k) const {
    return cR[((ti * T + tj) * (nR + 1) + n) * (KR + 1) + k];
  }
  double c_angular(int ti, int tj, int n, int k) const {
    return cA[((ti * T + tj) * (nA + 1) + n) * (KA + 1) + k];
  }
};

bool load_model(const oracle_model *p, Model &m) {
  if (!p) return false;
  m.T = p->n_types; m.nR = p->n_max_r; m.nA = p->n_max_a; m.KR = p->basis_r; m.KA = p->basis_a;
  m.l3 = p->l_max_3b; m.l4 = p->l_max_4b; m.l5 = p->l_max_5b; m.H = p->n_neuron;
  m.rcR = p->rc_r; m.rcA = p->rc_a;
  m.cR = p->c_r; m.cA = p->c_a; m.w0 = p->w0; m.b0 = p->b0; m.w1 = p->w1; m.b1 = p->b1;
  if (m.T < 1 || m.nR < 0 || m.nA < 0 || m.KR < 0 || m.KA < 0 || m.H < 1) return false;
  if (m.l3 < 1 || m.l3 > 4) return false;
  if (!(m.l4 == 0 || m.l4 == 2)) return false;
  if (!(m.l5 == 0 || m.l5 == 1)) return false;
  if (!(m.rcR > 0 && m.rcA > 0 && m.rcA <= m.rcR)) return false;
  if (!m.cR || !m.cA || !m.w0 || !m.b0 || !m.w1) return false;
  return true;
}

/* ---------------------------------------------------------------- Sec. II B */
/* Cosine cutoff f_c(r) (Sec. II B); the caller guarantees r < r_c. */
template <class R> R cutoff(const R &r, double rc) { return 0.5 * (1.0 + cos(PI * r / rc)); }

/* Basis f_k(r), k = 0..K, of Eq. f_n: one half of [T_k(2(r/r_c - 1)^2 - 1) + 1] times f_c,
 * with T_k the Chebyshev polynomials of the first kind (T_0 = 1, T_1 = x,
 * T_{k+1} = 2x T_k - T_{k-1}). */
template <class R> void basis(const R &r, double rc, int K, std::vector<R> &f) {
  R fc = cutoff(r, rc);
  R t = r / rc - 1.0;
  R x = 2.0 * t * t - 1.0;
  std::vector<R> Tk(K + 1);
  Tk[0] = R(1.0);
  if (K >= 1) Tk[1] = x;
  for (int k = 2; k <= K; ++k) Tk[k] = 2.0 * x * Tk[k - 1] - Tk[k - 2];
  f.assign(K + 1, R(0.0));
  for (int k = 0; k <= K; ++k) f[k] = 0.5 * (Tk[k] + 1.0) * fc;
}

/* ---------------------------------------------------------------- Sec. II D */
/* l of each of the 24 polynomials b_k. */
const int L_OF_K[24] = {1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 4};
/* Number of k used for l_max^3b = 1..4. */
const int K_END[5] = {0, 3, 8, 15, 24};

/* The 24 polynomials b_k(x, y, z) as printed in Sec. II D (with r^2 = x^2 + y^2 + z^2),
 * each divided by r^l, i.e. evaluated on the unit vector. */
template <class R> void angular_polynomials(const R &x, const R &y, const R &z, const R &r, R *b) {
  R r2 = x * x + y * y + z * z;
  R x2 = x * x, y2 = y * y, z2 = z * z;
  b[0] = z;
  b[1] = x;
  b[2] = y;
  b[3] = 3.0 * z2 - r2;
  b[4] = x * z;
  b[5] = y * z;
  b[6] = x2 - y2;
  b[7] = 2.0 * x * y;
  b[8] = (5.0 * z2 - 3.0 * r2) * z;
  b[9] = (5.0 * z2 - r2) * x;
  b[10] = (5.0 * z2 - r2) * y;
  b[11] = (x2 - y2) * z;
  b[12] = 2.0 * x * y * z;
  b[13] = (x2 - 3.0 * y2) * x;
  b[14] = (3.0 * x2 - y2) * y;
  b[15] = (35.0 * z2 - 30.0 * r2) * z2 + 3.0 * r2 * r2;
  b[16] = (7.0 * z2 - 3.0 * r2) * x * z;
  b[17] = (7.0 * z2 - 3.0 * r2) * y * z;
  b[18] = (7.0 * z2 - r2) * (x2 - y2);
  b[19] = (7.0 * z2 - r2) * 2.0 * x * y;
  b[20] = (x2 - 3.0 * y2) * x * z;
  b[21] = (3.0 * x2 - y2) * y * z;
  b[22] = (x2 - y2) * (x2 - y2) - 4.0 * x2 * y2;
  b[23] = 4.0 * (x2 - y2) * x * y;
  const R rpow[5] = {R(1.0), r, r * r, r * r * r, r * r * r * r};
  for (int k = 0; k < 24; ++k) b[k] = b[k] / rpow[L_OF_K[k]];
}

/* 3-body coefficients C3b_k as printed for q_n1 .. q_n4 (Sec. II D). */
void c3b(double *c) {
  c[0] = 0.25 * 3.0 / PI;
  c[1] = c[2] = 2.0 * 0.25 * 3.0 / (2.0 * PI);
  c[3] = (1.0 / 16.0) * 5.0 / PI;
  c[4] = c[5] = 2.0 * 0.25 * 15.0 / (2.0 * PI);
  c[6] = c[7] = 2.0 * (1.0 / 16.0) * 15.0 / (2.0 * PI);
  c[8] = (1.0 / 16.0) * 7.0 / PI;
  c[9] = c[10] = 2.0 * (1.0 / 64.0) * 21.0 / PI;
  c[11] = c[12] = 2.0 * (1.0 / 16.0) * 105.0 / (2.0 * PI);
  c[13] = c[14] = 2.0 * (1.0 / 64.0) * 35.0 / PI;
  c[15] = (9.0 / 256.0) * 1.0 / PI;
  c[16] = c[17] = 2.0 * (9.0 / 64.0) * 5.0 / PI;
  c[18] = c[19] = 2.0 * (9.0 / 64.0) * 5.0 / (2.0 * PI);
  c[20] = c[21] = 2.0 * (9.0 / 64.0) * 35.0 / PI;
  c[22] = c[23] = 2.0 * (9.0 / 256.0) * 35.0 / (2.0 * PI);
}

/* 4-body coefficients C4b_0..4 as printed for q_n222 (Sec. II D). */
void c4b(double *c) {
  double a20 = 0.25 * std::sqrt(5.0 / PI);        /* (1/4) sqrt(5/pi) */
  double a21 = 0.5 * std::sqrt(15.0 / (2.0 * PI)); /* (1/2) sqrt(15/(2 pi)) */
  double a22 = 0.25 * std::sqrt(15.0 / (2.0 * PI));/* (1/4) sqrt(15/(2 pi)) */
  c[0] = -std::sqrt(2.0 / 35.0) * a20 * a20 * a20;
  c[1] = -6.0 * std::sqrt(1.0 / 70.0) * a20 * a21 * a21;
  c[2] = 6.0 * std::sqrt(2.0 / 35.0) * a20 * a22 * a22;
  c[3] = 6.0 * std::sqrt(3.0 / 35.0) * a21 * a21 * a22;
  c[4] = -12.0 * std::sqrt(3.0 / 35.0) * a21 * a21 * a22;
}

/* 5-body coefficients C5b_0..2 as printed for q_n1111 (Sec. II D). */
void c5b(double *c) {
  c[0] = 21.0 / (80.0 * PI * PI);
  c[1] = 21.0 / (40.0 * PI * PI);
  c[2] = 21.0 / (80.0 * PI * PI);
}

/* ---------------------------------------------------------------- neighbours */
struct Cell {
  double H[3][3];    /* rows are the cell vectors */
  double Hinv[3][3]; /* s = r Hinv */
  double thick[3];   /* distance between opposite faces */
};

bool make_cell(const double *box, Cell &c) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) c.H[a][b] = box[3 * a + b];
  const double (*H)[3] = c.H;
  double cof[3][3];
  cof[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
  cof[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
  cof[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
  cof[1][0] = H[2][1] * H[0][2] - H[2][2] * H[0][1];
  cof[1][1] = H[2][2] * H[0][0] - H[2][0] * H[0][2];
  cof[1][2] = H[2][0] * H[0][1] - H[2][1] * H[0][0];
  cof[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
  cof[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
  cof[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];
  double det = H[0][0] * cof[0][0] + H[0][1] * cof[0][1] + H[0][2] * cof[0][2];
  if (!(std::fabs(det) > 0)) return false;
  /* inverse of H is cof^T / det */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) c.Hinv[a][b] = cof[b][a] / det;
  /* face distance along axis a = |det| / |row b x row c|; cof row a is that cross product */
  for (int a = 0; a < 3; ++a) {
    double n = std::sqrt(cof[a][0] * cof[a][0] + cof[a][1] * cof[a][1] + cof[a][2] * cof[a][2]);
    c.thick[a] = std::fabs(det) / n;
  }
  return true;
}

void to_frac(const Cell &c, const double *r, double *s) {
  for (int b = 0; b < 3; ++b) s[b] = r[0] * c.Hinv[0][b] + r[1] * c.Hinv[1][b] + r[2] * c.Hinv[2][b];
}

struct Pair {
  int j;
  int n[3];
  double d[3];
  double r;
};

/* All (j, n) with |r_j + n.H - r_i| < rc, (j, n) != (i, 0), in order of j then n. */
void find_neighbours(const Cell &c, int N, const double *pos, int i, double rc, std::vector<Pair> &out) {
  out.clear();
  double si[3];
  to_frac(c, pos + 3 * i, si);
  for (int j = 0; j < N; ++j) {
    double sj[3], ds[3];
    to_frac(c, pos + 3 * j, sj);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      ds[a] = sj[a] - si[a];
      double w = rc / c.thick[a];
      lo[a] = (int)std::floor(-w - ds[a]) - 1;
      hi[a] = (int)std::ceil(w - ds[a]) + 1;
    }
    for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
      for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
        for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
          if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
          Pair p;
          p.j = j;
          p.n[0] = n0; p.n[1] = n1; p.n[2] = n2;
          double r2 = 0;
          for (int b = 0; b < 3; ++b) {
            p.d[b] = (pos[3 * j + b] - pos[3 * i + b]) +
                     (n0 * c.H[0][b] + n1 * c.H[1][b] + n2 * c.H[2][b]);
            r2 += p.d[b] * p.d[b];
          }
          if (r2 < rc * rc) {
            p.r = std::sqrt(r2);
            out.push_back(p);
          }
        }
  }
}

/* ---------------------------------------------------------------- descriptor + ANN */
/* Descriptor q^i (Eqs. qin, g_n, f_n, S_nk and the explicit q_nl, q_n222, q_n1111) of an
 * atom of type ti whose neighbour pairs have types tj[p] and vectors d[p] (d = r_j - r_i). */
template <class R>
void descriptor(const Model &m, int ti, int np, const int *tj, const std::array<R, 3> *d, R *q) {
  const int D = m.ndes();
  for (int v = 0; v < D; ++v) q[v] = R(0.0);
  std::vector<R> f;
  /* radial components, Eq. qin */
  for (int p = 0; p < np; ++p) {
    R r = sqrt(d[p][0] * d[p][0] + d[p][1] * d[p][1] + d[p][2] * d[p][2]);
    if (!(value(r) < m.rcR)) continue;
    basis(r, m.rcR, m.KR, f);
    for (int n = 0; n <= m.nR; ++n) {
      R g(0.0);
      for (int k = 0; k <= m.KR; ++k) g += m.c_radial(ti, tj[p], n, k) * f[k];
      q[n] += g;
    }
  }
  /* angular sums, Eq. S_nk, with the angular cutoff r_c^A in g_n */
  std::vector<R> S((m.nA + 1) * 24, R(0.0));
  R b[24];
  for (int p = 0; p < np; ++p) {
    R r = sqrt(d[p][0] * d[p][0] + d[p][1] * d[p][1] + d[p][2] * d[p][2]);
    if (!(value(r) < m.rcA)) continue;
    basis(r, m.rcA, m.KA, f);
    angular_polynomials(d[p][0], d[p][1], d[p][2], r, b);
    for (int n = 0; n <= m.nA; ++n) {
      R g(0.0);
      for (int k = 0; k <= m.KA; ++k) g += m.c_angular(ti, tj[p], n, k) * f[k];
      for (int k = 0; k < 24; ++k) S[n * 24 + k] += g * b[k];
    }
  }
  double C3[24], C4[5], C5[3];
  c3b(C3);
  c4b(C4);
  c5b(C5);
  int off = m.nR + 1;
  for (int l = 1; l <= m.l3; ++l) {
    for (int n = 0; n <= m.nA; ++n) {
      R acc(0.0);
      for (int k = K_END[l - 1]; k < K_END[l]; ++k) acc += C3[k] * S[n * 24 + k] * S[n * 24 + k];
      q[off + n] = acc;
    }
    off += m.nA + 1;
  }
  if (m.l4 >= 2) {
    for (int n = 0; n <= m.nA; ++n) {
      const R *s = &S[n * 24];
      q[off + n] = C4[0] * s[3] * s[3] * s[3] + C4[1] * s[3] * (s[4] * s[4] + s[5] * s[5]) +
                   C4[2] * s[3] * (s[6] * s[6] + s[7] * s[7]) + C4[3] * s[6] * (s[5] * s[5] - s[4] * s[4]) +
                   C4[4] * s[4] * s[5] * s[7];
    }
    off += m.nA + 1;
  }
  if (m.l5 >= 1) {
    for (int n = 0; n <= m.nA; ++n) {
      const R *s = &S[n * 24];
      R s12 = s[1] * s[1] + s[2] * s[2];
      q[off + n] = C5[0] * s[0] * s[0] * s[0] * s[0] + C5[1] * s[0] * s[0] * s12 + C5[2] * s12 * s12;
    }
    off += m.nA + 1;
  }
}

/* Site energy of Eq. Ui: sum_mu w1_mu tanh(sum_nu w0_{mu nu} q_nu - b0_mu) - b1. */
template <class R> R site_energy(const Model &m, const R *q) {
  const int D = m.ndes();
  R U(0.0);
  for (int mu = 0; mu < m.H; ++mu) {
    R z(0.0);
    for (int nu = 0; nu < D; ++nu) z += m.w0[mu * D + nu] * q[nu];
    U += m.w1[mu] * tanh(z - m.b0[mu]);
  }
  return U - m.b1;
}

/* Neighbourhood of one atom: pairs within r_c^R, their types and vectors. */
struct Env {
  std::vector<Pair> pairs;
  std::vector<int> tj;
};

double site_energy_of(const Model &m, int ti, const Env &e) {
  const int np = (int)e.pairs.size();
  std::vector<std::array<double, 3>> d(np);
  for (int p = 0; p < np; ++p)
    for (int c = 0; c < 3; ++c) d[p][c] = e.pairs[p].d[c];
  std::vector<double> q(m.ndes());
  descriptor<double>(m, ti, np, e.tj.data(), d.data(), q.data());
  return site_energy<double>(m, q.data());
}

/* Partial forces dU_i/dr_ij (Eq. partial_force) for every pair of the neighbourhood:
 * forward-mode derivative of U_i with the pair vector of pair p as the seed. */
void partial_forces(const Model &m, int ti, const Env &e, std::vector<std::array<double, 3>> &P) {
  const int np = (int)e.pairs.size();
  P.assign(np, {0.0, 0.0, 0.0});
  std::vector<std::array<Dual, 3>> d(np);
  std::vector<Dual> q(m.ndes());
  for (int p = 0; p < np; ++p) {
    for (int a = 0; a < np; ++a)
      for (int c = 0; c < 3; ++c) d[a][c] = Dual(e.pairs[a].d[c]);
    for (int c = 0; c < 3; ++c) d[p][c].g[c] = 1.0;
    descriptor<Dual>(m, ti, np, e.tj.data(), d.data(), q.data());
    Dual U = site_energy<Dual>(m, q.data());
    for (int c = 0; c < 3; ++c) P[p][c] = U.g[c];
  }
}

int threads_or_default(int n_threads) {
#ifdef _OPENMP
  return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
  (void)n_threads;
  return 1;
#endif
}

/* Forces and virials of the atoms in `sel` (all atoms when sel is null) from the partial
 * forces of each selected atom and of each of its neighbours (Eqs. F_ij, F_i, virial). */
int compute(const Model &m, int N, const double *pos, const int *types, const Cell &cell, int n_sel,
            const int *sel, double *U_out, double *F_out, double *W_out, int n_threads) {
  std::vector<int> selected;
  if (sel) selected.assign(sel, sel + n_sel);
  else {
    selected.resize(N);
    for (int i = 0; i < N; ++i) selected[i] = i;
  }
  for (int i : selected)
    if (i < 0 || i >= N) return -1;
  for (int i = 0; i < N; ++i)
    if (types[i] < 0 || types[i] >= m.T) return -1;
  const int nt = threads_or_default(n_threads);
  /* neighbourhoods of the selected atoms */
  std::vector<int> slot(N, -1);
  std::vector<int> need;
  for (int i : selected)
    if (slot[i] < 0) { slot[i] = (int)need.size(); need.push_back(i); }
  std::vector<Env> env(need.size());
  const int n_first = (int)need.size();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int a = 0; a < n_first; ++a) find_neighbours(cell, N, pos, need[a], m.rcR, env[a].pairs);
  /* ...and of every neighbour of a selected atom */
  for (int a = 0; a < n_first; ++a)
    for (const Pair &p : env[a].pairs)
      if (slot[p.j] < 0) { slot[p.j] = (int)need.size(); need.push_back(p.j); }
  env.resize(need.size());
  const int n_need = (int)need.size();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int a = n_first; a < n_need; ++a) find_neighbours(cell, N, pos, need[a], m.rcR, env[a].pairs);
  for (int a = 0; a < n_need; ++a) {
    env[a].tj.resize(env[a].pairs.size());
    for (size_t p = 0; p < env[a].pairs.size(); ++p) env[a].tj[p] = types[env[a].pairs[p].j];
  }
  /* partial forces of every needed atom */
  std::vector<std::vector<std::array<double, 3>>> P(n_need);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int a = 0; a < n_need; ++a) partial_forces(m, types[need[a]], env[a], P[a]);
  /* assemble */
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int s = 0; s < (int)selected.size(); ++s) {
    const int i = selected[s];
    const int a = slot[i];
    if (U_out) U_out[s] = site_energy_of(m, types[i], env[a]);
    double F[3] = {0, 0, 0}, W[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (size_t p = 0; p < env[a].pairs.size(); ++p) {
      const Pair &pr = env[a].pairs[p];
      const int b = slot[pr.j];
      /* dU_j/dr_ji: the pair (i, -n) in the neighbourhood of j */
      double Pji[3] = {0, 0, 0};
      for (size_t q = 0; q < env[b].pairs.size(); ++q) {
        const Pair &rq = env[b].pairs[q];
        if (rq.j == i && rq.n[0] == -pr.n[0] && rq.n[1] == -pr.n[1] && rq.n[2] == -pr.n[2]) {
          for (int c = 0; c < 3; ++c) Pji[c] = P[b][q][c];
          break;
        }
      }
      for (int c = 0; c < 3; ++c) F[c] += P[a][p][c] - Pji[c];
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) W[x][y] += pr.d[x] * Pji[y];
    }
    if (F_out)
      for (int c = 0; c < 3; ++c) F_out[3 * s + c] = F[c];
    if (W_out) {
      /* component order xx, yy, zz, xy, xz, yz, yx, zx, zy */
      const int ord[9][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}, {1, 0}, {2, 0}, {2, 1}};
      for (int c = 0; c < 9; ++c) W_out[9 * s + c] = W[ord[c][0]][ord[c][1]];
    }
  }
  return 0;
}

/* Total heat current in the form of Eq. J-2: J = -sum_i sum_(j,n) r_ij (dU_i/dr_ij . v_j),
 * from every atom's own partial forces and its neighbours' velocities. */
int heat_current_j2(const Model &m, int N, const double *pos, const int *types, const Cell &cell, const double *vel,
                    double *J, int n_threads) {
  for (int i = 0; i < N; ++i)
    if (types[i] < 0 || types[i] >= m.T) return -1;
  const int nt = threads_or_default(n_threads);
  std::vector<Env> env(N);
  std::vector<std::array<double, 3>> part((size_t)N);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int i = 0; i < N; ++i) {
    find_neighbours(cell, N, pos, i, m.rcR, env[i].pairs);
    env[i].tj.resize(env[i].pairs.size());
    for (size_t p = 0; p < env[i].pairs.size(); ++p) env[i].tj[p] = types[env[i].pairs[p].j];
    std::vector<std::array<double, 3>> P;
    partial_forces(m, types[i], env[i], P);
    double acc[3] = {0, 0, 0};
    for (size_t p = 0; p < env[i].pairs.size(); ++p) {
      const Pair &pr = env[i].pairs[p];
      const double *vj = vel + 3 * (size_t)pr.j;
      const double dot = P[p][0] * vj[0] + P[p][1] * vj[1] + P[p][2] * vj[2];
      for (int c = 0; c < 3; ++c) acc[c] -= pr.d[c] * dot;
    }
    for (int c = 0; c < 3; ++c) part[i][c] = acc[c];
  }
  for (int c = 0; c < 3; ++c) J[c] = 0.0;
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) J[c] += part[i][c];
  return 0;
}

}  // namespace

/* ==================================================================== C entry points */
extern "C" {

/* Descriptor length N_des. */
int oracle_n_des(const oracle_model *pm) {
  Model m;
  if (!load_model(pm, m)) return -1;
  return m.ndes();
}

/* f_k(r), k = 0..K, of Eq. f_n (zero for r >= rc). */
void oracle_radial_basis(double rc, int K, double r, double *f) {
  if (!(r < rc)) {
    for (int k = 0; k <= K; ++k) f[k] = 0.0;
    return;
  }
  std::vector<double> v;
  basis<double>(r, rc, K, v);
  for (int k = 0; k <= K; ++k) f[k] = v[k];
}

/* The 24 angular polynomials b_k / r^l for the vector (x, y, z). */
void oracle_angular_polynomials(double x, double y, double z, double *b) {
  double r = std::sqrt(x * x + y * y + z * z);
  angular_polynomials<double>(x, y, z, r, b);
}

/* Number of neighbours within rc of every atom (brute force over all images). */
int oracle_neighbor_counts(int N, const double *pos, const double *box, double rc, int *counts) {
  Cell c;
  if (N < 0 || !make_cell(box, c) || !(rc > 0)) return -1;
  std::vector<Pair> tmp;
  for (int i = 0; i < N; ++i) {
    find_neighbours(c, N, pos, i, rc, tmp);
    counts[i] = (int)tmp.size();
  }
  return 0;
}

/* Neighbours (j, image shift n, vector d) within rc of atom i; returns the count, or -1. At
 * most `cap` entries are written. */
int oracle_neighbors(int N, const double *pos, const double *box, double rc, int i, int cap, int *j_out,
                     int *n_out, double *d_out) {
  Cell c;
  if (N < 1 || i < 0 || i >= N || !make_cell(box, c)) return -1;
  std::vector<Pair> tmp;
  find_neighbours(c, N, pos, i, rc, tmp);
  for (int p = 0; p < (int)tmp.size() && p < cap; ++p) {
    j_out[p] = tmp[p].j;
    for (int a = 0; a < 3; ++a) {
      n_out[3 * p + a] = tmp[p].n[a];
      d_out[3 * p + a] = tmp[p].d[a];
    }
  }
  return (int)tmp.size();
}

/* Descriptor vectors q^i [n_sel][N_des] of the selected atoms (all when sel is null). */
int oracle_descriptors(const oracle_model *pm, int N, const double *pos, const int *types, const double *box,
                       int n_sel, const int *sel, double *q_out, int n_threads) {
  Model m;
  Cell c;
  if (!load_model(pm, m) || N < 0 || !make_cell(box, c)) return -1;
  const int ns = sel ? n_sel : N;
  const int D = m.ndes();
  const int nt = threads_or_default(n_threads);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : bad)
  for (int s = 0; s < ns; ++s) {
    const int i = sel ? sel[s] : s;
    if (i < 0 || i >= N || types[i] < 0 || types[i] >= m.T) { bad |= 1; continue; }
    Env e;
    find_neighbours(c, N, pos, i, m.rcR, e.pairs);
    const int np = (int)e.pairs.size();
    std::vector<int> tj(np);
    std::vector<std::array<double, 3>> d(np);
    for (int p = 0; p < np; ++p) {
      tj[p] = types[e.pairs[p].j];
      for (int a = 0; a < 3; ++a) d[p][a] = e.pairs[p].d[a];
    }
    descriptor<double>(m, types[i], np, tj.data(), d.data(), q_out + (size_t)s * D);
  }
  return bad ? -1 : 0;
}

/* Site energy (Eq. Ui) of one descriptor vector. */
int oracle_ann(const oracle_model *pm, const double *q, double *U) {
  Model m;
  if (!load_model(pm, m)) return -1;
  *U = site_energy<double>(m, q);
  return 0;
}

/* Site energies U [n_sel], forces F [n_sel][3] and per-atom virials W [n_sel][9]
 * (xx, yy, zz, xy, xz, yz, yx, zx, zy) of the selected atoms (all when sel is null).
 * Any output pointer may be null. */
int oracle_compute(const oracle_model *pm, int N, const double *pos, const int *types, const double *box,
                   int n_sel, const int *sel, double *U, double *F, double *W, int n_threads) {
  Model m;
  Cell c;
  if (!load_model(pm, m) || N < 0 || !make_cell(box, c)) return -1;
  if (N == 0) return 0;
  return compute(m, N, pos, types, c, sel ? n_sel : N, sel, U, F, W, n_threads);
}

/* Velocity-Verlet NVE: v += dt/2 a; x += dt v; wrap into the cell; recompute F; v += dt/2 a,
 * with a = F / (m * 103.6427...) in Angstrom/fs^2 (eV, Angstrom, fs, u). pos and vel are
 * updated in place; thermo [n_steps+1][3] receives (E_pot, E_kin, T) after each step
 * (row 0 = initial state); force_out [N][3] receives the final forces. */
int oracle_md(const oracle_model *pm, int N, double *pos, double *vel, const int *types, const double *mass,
              const double *box, int n_steps, double dt, double *thermo, double *force_out, int n_threads) {
  Model m;
  Cell c;
  if (!load_model(pm, m) || N < 1 || !make_cell(box, c) || n_steps < 0) return -1;
  const double ev_j = 1.602176634e-19, amu_kg = 1.66053906660e-27;
  const double kappa = amu_kg * 1e-20 / 1e-30 / ev_j; /* u A^2 / fs^2 in eV */
  const double kB = 8.617333262e-5;
  std::vector<double> U(N), F(3 * (size_t)N);
  auto evaluate = [&](double *epot) {
    int rc = compute(m, N, pos, types, c, N, nullptr, U.data(), F.data(), nullptr, n_threads);
    double e = 0;
    for (int i = 0; i < N; ++i) e += U[i];
    *epot = e;
    return rc;
  };
  auto record = [&](int s, double epot) {
    if (!thermo) return;
    double ke = 0;
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) ke += 0.5 * kappa * mass[types[i]] * vel[3 * i + a] * vel[3 * i + a];
    thermo[3 * s + 0] = epot;
    thermo[3 * s + 1] = ke;
    thermo[3 * s + 2] = N > 1 ? 2.0 * ke / ((3.0 * N - 3.0) * kB) : 0.0;
  };
  double epot;
  if (evaluate(&epot)) return -1;
  record(0, epot);
  for (int s = 1; s <= n_steps; ++s) {
    for (int i = 0; i < N; ++i) {
      const double inv = 1.0 / (mass[types[i]] * kappa);
      for (int a = 0; a < 3; ++a) {
        vel[3 * i + a] += 0.5 * dt * F[3 * i + a] * inv;
        pos[3 * i + a] += dt * vel[3 * i + a];
      }
      double sf[3];
      to_frac(c, pos + 3 * i, sf);
      for (int a = 0; a < 3; ++a) sf[a] -= std::floor(sf[a]);
      for (int a = 0; a < 3; ++a) pos[3 * i + a] = sf[0] * c.H[0][a] + sf[1] * c.H[1][a] + sf[2] * c.H[2][a];
    }
    if (evaluate(&epot)) return -1;
    for (int i = 0; i < N; ++i) {
      const double inv = 1.0 / (mass[types[i]] * kappa);
      for (int a = 0; a < 3; ++a) vel[3 * i + a] += 0.5 * dt * F[3 * i + a] * inv;
    }
    record(s, epot);
  }
  if (force_out) std::memcpy(force_out, F.data(), sizeof(double) * 3 * (size_t)N);
  return 0;
}

/* Number of OpenMP threads a call with n_threads <= 0 uses. */
int oracle_max_threads(void) { return threads_or_default(0); }

/* Total heat current by Eq. J-2 (vel [N][3] in Angstrom/fs; J [3] in eV Angstrom/fs). */
int oracle_heat_current_j2(const oracle_model *pm, int N, const double *pos, const int *types, const double *box,
                           const double *vel, double *J, int n_threads) {
  Model m;
  Cell c;
  if (!load_model(pm, m) || N < 1 || !make_cell(box, c)) return -1;
  return heat_current_j2(m, N, pos, types, c, vel, J, n_threads);
}

}  // extern "C"
