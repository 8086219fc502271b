// Hermite-4 device routines (Sec. 2.2.1, Eqs. 3-4, Algorithm 2) for sm_103a.
//
// FP64 is the scarce resource on this chip (2 DFMA per clock per SM, i.e. half a lane
// per clock on each of the 4 SM sub-partitions; DADD/DMUL issue ~1.2x slower than DFMA;
// rsqrt(double) ~ 6 DFMA slots).  The routines below therefore
//  - evaluate every unordered pair once (acceleration and jerk of both bodies),
//  - keep the corrector in FMA form with step-invariant bases precomputed per step,
//  - do the monitor's tests with bounds that skip square roots in the common case,
//  - keep no lane idle that can be avoided.
#pragma once
#include "common.cuh"

namespace swarm {

// Coefficients of one step of length h.
struct HCoef {
  double h, h2_2, h3_6, hh, h2_12;
};
__device__ __forceinline__ HCoef hcoef(double h) {
  HCoef c;
  c.h = h;
  c.h2_2 = 0.5 * h * h;
  c.h3_6 = c.h2_2 * h * (1.0 / 3.0);
  c.hh = 0.5 * h;
  c.h2_12 = h * h * (1.0 / 12.0);
  return c;
}
// the same coefficients with the products in DFMA form (steps chosen per step)
__device__ __forceinline__ HCoef hcoef(const F64k &k, double h) {
  HCoef c;
  c.h = h;
  c.h2_2 = kmul(k, kmul(k, 0.5, h), h);
  c.h3_6 = kmul(k, kmul(k, c.h2_2, h), 1.0 / 3.0);
  c.hh = kmul(k, 0.5, h);
  c.h2_12 = kmul(k, kmul(k, h, h), 1.0 / 12.0);
  return c;
}
// Printed-form corrector (Eq. 4 with 3/20 and the predicted base): its velocity update
// equals the time-symmetric one, its position update is
//   x_{k+1} = XP + (3/20) h^2 a_k - (1/30) h^3 j_k,  XP = x_p - (3/20) h^2 a0 - (7/60) h^3 j0.
struct PCoef {
  double pa, pj, ca, cj;
};
__device__ __forceinline__ PCoef pcoef(double h) {
  PCoef c;
  const double h2 = h * h, h3 = h2 * h;
  c.pa = -0.15 * h2;
  c.pj = -(7.0 / 60.0) * h3;
  c.ca = 0.15 * h2;
  c.cj = -(1.0 / 30.0) * h3;
  return c;
}
__device__ __forceinline__ HCoef hsel(bool p, const HCoef &a, const HCoef &b) {
  HCoef c;
  c.h = p ? a.h : b.h;
  c.h2_2 = p ? a.h2_2 : b.h2_2;
  c.h3_6 = p ? a.h3_6 : b.h3_6;
  c.hh = p ? a.hh : b.hh;
  c.h2_12 = p ? a.h2_12 : b.h2_12;
  return c;
}

// Geometry of one pair, from body i to body j (Eq. 1 and its time derivative):
//   dx = x_j - x_i, dv = v_j - v_i, rho = 1/|dx|,
//   w  = dv - 3 (dx.dv)/|dx|^2 dx   so that   a_i += m_j rho^3 dx,  jerk_i += m_j rho^3 w
// and the partner receives the opposite terms scaled by m_i.
// Products and differences in the DFMA forms of `kmul` / `ksub` (same values).
__device__ __forceinline__ void pair_geom(const F64k &k, const double (&xi)[3], const double (&vi)[3],
                                          const double (&xj)[3], const double (&vj)[3], double (&dx)[3],
                                          double (&w)[3], double &rho3, double &r2) {
  double dv[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    dx[c] = ksub(k, xj[c], xi[c]);
    dv[c] = ksub(k, vj[c], vi[c]);
  }
  r2 = kmul(k, dx[0], dx[0]);
  r2 = fma(dx[1], dx[1], r2);
  r2 = fma(dx[2], dx[2], r2);
  double rv = kmul(k, dx[0], dv[0]);
  rv = fma(dx[1], dv[1], rv);
  rv = fma(dx[2], dv[2], rv);
  double rho = rsqrt(r2);
  double rho2 = kmul(k, rho, rho);
  rho3 = kmul(k, rho2, rho);
  double cc = kmul(k, -3.0, kmul(k, rv, rho2));
#pragma unroll
  for (int c = 0; c < 3; c++) w[c] = fma(cc, dx[c], dv[c]);
}

// ---------------------------------------------------------------- group collectives
// All lanes of the warp execute these (full-mask shuffles); each group of N lanes
// starting at `base` reduces its own values.
template <int N>
__device__ __forceinline__ double grp_sum(double val, int b, int base) {
  // segmented tree: after the loop lane b = 0 of the group holds the sum
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, val, off);
    val += (b + off < N) ? o : 0.0;
  }
  return shfl(val, base);
}

// the same sum with the additions as DFMA
template <int N>
__device__ __forceinline__ double grp_sum(const F64k &k, double val, int b, int base) {
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, val, off);
    val = kadd(k, (b + off < N) ? o : 0.0, val);
  }
  return shfl(val, base);
}

// exclusive prefix sum over the group (lane b gets the sum over lanes 0..b-1)
template <int N>
__device__ __forceinline__ double grp_scan_excl(double val, int b) {
  double inc = val;
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_up_sync(0xffffffffu, inc, off);
    inc += (b >= off) ? o : 0.0;
  }
  double ex = __shfl_up_sync(0xffffffffu, inc, 1);
  return b > 0 ? ex : 0.0;
}

template <int N>
__device__ __forceinline__ double grp_scan_excl(const F64k &k, double val, int b) {
  double inc = val;
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_up_sync(0xffffffffu, inc, off);
    inc = kadd(k, (b >= off) ? o : 0.0, inc);
  }
  double ex = __shfl_up_sync(0xffffffffu, inc, 1);
  return b > 0 ? ex : 0.0;
}

// exclusive suffix sum (lane b gets the sum over lanes b+1..N-1)
template <int N>
__device__ __forceinline__ double grp_suffix_excl(double val, int b) {
  double inc = val;
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, inc, off);
    inc += (b + off < N) ? o : 0.0;
  }
  double ex = __shfl_down_sync(0xffffffffu, inc, 1);
  return b + 1 < N ? ex : 0.0;
}

// ---------------------------------------------------------------- body per lane ("ring")
// Lanes g*N .. g*N+N-1 of a warp hold the N bodies of system g.  In round r = 1..(N-1)/2
// lane b evaluates the pair (b, b+r mod N) and hands the partner's share of the pair back
// to lane b+r by shuffle; for even N a last round r = N/2 has both lanes of each pair take
// their own share.  Every unordered pair is evaluated exactly once per full round set.
template <int N>
struct Ring {
  static constexpr int G = 32 / N;             // systems per warp
  static constexpr int RF = (N - 1) / 2;       // full rounds (with reaction)
  static constexpr bool HALF = (N % 2) == 0;   // extra self-sufficient round
  static constexpr int RT = RF + (HALF ? 1 : 0);
};

// MON: also return q2 (squared distance of this body to body 0) and d2[r] (squared
// distance of this lane's pair in round r) for the monitor.
template <int N, bool MON>
__device__ __forceinline__ void ring_accjerk(const F64k &k, const double (&x)[3], const double (&v)[3], double m, int b, int base,
                                             double (&a)[3], double (&jk)[3], double &q2,
                                             double (&d2)[Ring<N>::RT > 0 ? Ring<N>::RT : 1]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    a[c] = 0.0;
    jk[c] = 0.0;
  }
  q2 = 0.0;
#pragma unroll
  for (int r = 1; r <= Ring<N>::RF; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    int q = b - r;
    if (q < 0) q += N;
    double xj[3], vj[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xj[c] = shfl(x[c], base + p);
      vj[c] = shfl(v[c], base + p);
    }
    double mj = shfl(m, base + p);
    double dx[3], w[3], rho3, r2;
    pair_geom(k, x, v, xj, vj, dx, w, rho3, r2);
    double sj = kmul(k, mj, rho3);
    double si = kmul(k, m, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[c] = fma(sj, dx[c], a[c]);
      jk[c] = fma(sj, w[c], jk[c]);
    }
    // reaction from lane q, which evaluated the pair (q, b)
    double rdx[3], rw[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      rdx[c] = shfl(dx[c], base + q);
      rw[c] = shfl(w[c], base + q);
    }
    double rs = shfl(si, base + q);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[c] = fma(-rs, rdx[c], a[c]);
      jk[c] = fma(-rs, rw[c], jk[c]);
    }
    if (MON) {
      double rr2 = shfl(r2, base + q);
      d2[r - 1] = r2;
      if (p == 0) q2 = r2;
      if (q == 0) q2 = rr2;
    }
  }
  if (Ring<N>::HALF) {
    constexpr int r = N / 2;
    int p = b + r;
    if (p >= N) p -= N;
    double xj[3], vj[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xj[c] = shfl(x[c], base + p);
      vj[c] = shfl(v[c], base + p);
    }
    double mj = shfl(m, base + p);
    double dx[3], w[3], rho3, r2;
    pair_geom(k, x, v, xj, vj, dx, w, rho3, r2);
    double sj = kmul(k, mj, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[c] = fma(sj, dx[c], a[c]);
      jk[c] = fma(sj, w[c], jk[c]);
    }
    if (MON) {
      d2[Ring<N>::RT - 1] = r2;
      if (p == 0) q2 = r2;
    }
  }
}

// Energy (Eq. 6, pairs once) and angular momentum of the lane's system, valid in the
// group's first lane.  Only called at log points.
template <int N>
__device__ __forceinline__ void ring_energy(const double (&x)[3], const double (&v)[3], double m, int b, int base,
                                            double (&out)[4]) {
  double e = 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double L0 = m * (x[1] * v[2] - x[2] * v[1]);
  double L1 = m * (x[2] * v[0] - x[0] * v[2]);
  double L2 = m * (x[0] * v[1] - x[1] * v[0]);
#pragma unroll
  for (int r = 1; r <= N / 2; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    double d0 = shfl(x[0], base + p) - x[0];
    double d1 = shfl(x[1], base + p) - x[1];
    double d2 = shfl(x[2], base + p) - x[2];
    double mp = shfl(m, base + p);
    double pot = m * mp * rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (Ring<N>::HALF && r == N / 2) pot *= 0.5;  // both lanes of the pair count it
    e -= pot;
  }
  double s[4] = {e, L0, L1, L2};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    double tot = s[k];
#pragma unroll
    for (int j = 1; j < N; j++) tot += shfl(s[k], base + j);
    out[k] = tot;
  }
  // out[] is the sum over the group only in the group's lane 0 (base + 0 reads base + j);
  // the other lanes hold partial sums that are not used.
}

// ---------------------------------------------------------------- system per lane
// One lane integrates a whole system held in registers; pairs in the order
// planet-planet first, then star-planet, so every body's star term comes last (Sec. 4.2).
template <int N>
__device__ __forceinline__ void spl_accjerk(const F64k &kk, const double (&x)[N][3], const double (&v)[N][3], const double (&m)[N],
                                            double (&a)[N][3], double (&jk)[N][3], double (&q2)[N],
                                            double (&d2)[N][N]) {
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[i][c] = 0.0;
      jk[i][c] = 0.0;
    }
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) {
      double dx[3], w[3], rho3, r2;
      pair_geom(kk, x[i], v[i], x[k], v[k], dx, w, rho3, r2);
      double sk = kmul(kk, m[k], rho3), si = kmul(kk, m[i], rho3);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        a[i][c] = fma(sk, dx[c], a[i][c]);
        jk[i][c] = fma(sk, w[c], jk[i][c]);
        a[k][c] = fma(-si, dx[c], a[k][c]);
        jk[k][c] = fma(-si, w[c], jk[k][c]);
      }
      d2[i][k] = r2;
    }
#pragma unroll
  for (int k = 1; k < N; k++) {
    double dx[3], w[3], rho3, r2;
    pair_geom(kk, x[0], v[0], x[k], v[k], dx, w, rho3, r2);
    double sk = kmul(kk, m[k], rho3), s0 = kmul(kk, m[0], rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[0][c] = fma(sk, dx[c], a[0][c]);
      jk[0][c] = fma(sk, w[c], jk[0][c]);
      a[k][c] = fma(-s0, dx[c], a[k][c]);
      jk[k][c] = fma(-s0, w[c], jk[k][c]);
    }
    q2[k] = r2;
  }
}

// Coordinates relative to body 0 (k >= 1, in place) and the barycentre of the system, and
// back: x_0 = X_cm - sum_{k>=1} m_k X_k / M, x_k = X_k + x_0 (likewise v).
template <int N>
__device__ __forceinline__ void spl_to_rel(const double (&m)[N], double (&x)[N][3], double (&v)[N][3], double &Minv,
                                           double (&Xc)[3], double (&Vc)[3]) {
  double Mt = m[0];
#pragma unroll
  for (int i = 1; i < N; i++) Mt += m[i];
  Minv = 1.0 / Mt;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double sx = m[0] * x[0][c], sv = m[0] * v[0][c];
#pragma unroll
    for (int i = 1; i < N; i++) {
      sx = fma(m[i], x[i][c], sx);
      sv = fma(m[i], v[i][c], sv);
    }
    Xc[c] = sx * Minv;
    Vc[c] = sv * Minv;
#pragma unroll
    for (int k = 1; k < N; k++) {
      x[k][c] -= x[0][c];
      v[k][c] -= v[0][c];
    }
  }
}

template <int N>
__device__ __forceinline__ void spl_from_rel(const double (&m)[N], const double (&x)[N][3], const double (&v)[N][3],
                                             double Minv, const double (&Xc)[3], const double (&Vc)[3],
                                             double (&xo)[N][3], double (&vo)[N][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double sx = 0.0, sv = 0.0;
#pragma unroll
    for (int k = 1; k < N; k++) {
      sx = fma(m[k], x[k][c], sx);
      sv = fma(m[k], v[k][c], sv);
    }
    const double x0 = fma(-sx, Minv, Xc[c]), v0 = fma(-sv, Minv, Vc[c]);
    xo[0][c] = x0;
    vo[0][c] = v0;
#pragma unroll
    for (int k = 1; k < N; k++) {
      xo[k][c] = x[k][c] + x0;
      vo[k][c] = v[k][c] + v0;
    }
  }
}

// Acceleration and jerk of bodies k = 1..N-1 relative to body 0 (index 0: body 0 itself), from
// the coordinates X_k = x_k - x_0, V_k = v_k - v_0 (Eq. 1 and its time derivative):
//   A_k = a_k - a_0 = -m_0 s_k X_k - I + sum_{i >= 1, i != k} m_i s_ik (X_i - X_k),
//   I = a_0 = sum_{j >= 1} m_j s_j X_j,   s = 1/r^3,
// and J_k likewise with the jerk vectors w of the pairs; A[0], J[0] receive body 0's own
// acceleration and jerk, I and its jerk counterpart.  Monitor distances:
// q2[k] = |X_k|^2, d2[i][k] = |X_k - X_i|^2.
template <int N>
__device__ __forceinline__ void spl_accjerk_rel(const F64k &kk, const double (&X)[N][3], const double (&V)[N][3],
                                                const double (&m)[N], double (&A)[N][3], double (&J)[N][3],
                                                double (&q2)[N], double (&d2)[N][N]) {
  double w0[N][3], m0s[N], IA[3], IJ[3];
#pragma unroll
  for (int k = 1; k < N; k++) {
    double r2 = kmul(kk, X[k][0], X[k][0]);
    r2 = fma(X[k][1], X[k][1], r2);
    r2 = fma(X[k][2], X[k][2], r2);
    double rv = kmul(kk, X[k][0], V[k][0]);
    rv = fma(X[k][1], V[k][1], rv);
    rv = fma(X[k][2], V[k][2], rv);
    const double rho = rsqrt(r2);
    const double rho2 = kmul(kk, rho, rho);
    const double s3 = kmul(kk, rho2, rho);
    const double cc = kmul(kk, -3.0, kmul(kk, rv, rho2));
    const double ms = kmul(kk, m[k], s3);
    m0s[k] = kmul(kk, m[0], s3);
    q2[k] = r2;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      w0[k][c] = fma(cc, X[k][c], V[k][c]);
      IA[c] = k == 1 ? kmul(kk, ms, X[k][c]) : fma(ms, X[k][c], IA[c]);
      IJ[c] = k == 1 ? kmul(kk, ms, w0[k][c]) : fma(ms, w0[k][c], IJ[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    A[0][c] = IA[c];
    J[0][c] = IJ[c];
  }
#pragma unroll
  for (int k = 1; k < N; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      A[k][c] = fma(-m0s[k], X[k][c], -IA[c]);
      J[k][c] = fma(-m0s[k], w0[k][c], -IJ[c]);
    }
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) {
      double dx[3], w[3], rho3, r2;
      pair_geom(kk, X[i], V[i], X[k], V[k], dx, w, rho3, r2);
      const double sk = kmul(kk, m[k], rho3), si = kmul(kk, m[i], rho3);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        A[i][c] = fma(sk, dx[c], A[i][c]);
        J[i][c] = fma(sk, w[c], J[i][c]);
        A[k][c] = fma(-si, dx[c], A[k][c]);
        J[k][c] = fma(-si, w[c], J[k][c]);
      }
      d2[i][k] = r2;
    }
}

// 1/|d| and its square for each pair of a system per lane (index [0][k]: body 0 with body
// k; [i][k], 1 <= i < k: bodies i and k), kept from one evaluation of a step to the next.
template <int N>
struct RhoCache {
  double r[N][N], r2[N][N];
};

// rsqrt out of line: the rare branch of spl_accjerk_rel_cached
static __device__ __noinline__ double rsqrt_call(double x) { return rsqrt(x); }

// spl_accjerk_rel for the evaluations of a step after its first: the positions have moved
// by the corrector only, so each 1/|d| follows from the previous evaluation's value rho_o
// by the series of (1 + delta)^(-1/2), delta = |d|^2 rho_o^2 - 1:
//   rho = rho_o (1 - delta/2 + 3 delta^2/8),  error 5|delta|^3/16,
// taken when |delta| < 2^-20 for every pair of the lane (error below 2.9e-19; on the
// 131072 x 3 ensemble delta ~ 1e-10), else rsqrt.  FIRST: the step's first evaluation
// (rsqrt, filling the cache).  Same outputs as spl_accjerk_rel.
template <int N, bool FIRST>
__device__ __forceinline__ void spl_accjerk_rel_cached(const F64k &kk, const double (&X)[N][3],
                                                       const double (&V)[N][3], const double (&m)[N],
                                                       double (&A)[N][3], double (&J)[N][3], double (&q2)[N],
                                                       double (&d2)[N][N], RhoCache<N> &rc) {
  // geometry of every pair
  double rv[N][N], dx[N][N][3], dv[N][N][3], rho[N][N];
#pragma unroll
  for (int k = 1; k < N; k++) {
    double r2 = kmul(kk, X[k][0], X[k][0]);
    r2 = fma(X[k][1], X[k][1], r2);
    r2 = fma(X[k][2], X[k][2], r2);
    double t = kmul(kk, X[k][0], V[k][0]);
    t = fma(X[k][1], V[k][1], t);
    rv[0][k] = fma(X[k][2], V[k][2], t);
    q2[k] = r2;
  }
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        dx[i][k][c] = ksub(kk, X[k][c], X[i][c]);
        dv[i][k][c] = ksub(kk, V[k][c], V[i][c]);
      }
      double r2 = kmul(kk, dx[i][k][0], dx[i][k][0]);
      r2 = fma(dx[i][k][1], dx[i][k][1], r2);
      r2 = fma(dx[i][k][2], dx[i][k][2], r2);
      double t = kmul(kk, dx[i][k][0], dv[i][k][0]);
      t = fma(dx[i][k][1], dv[i][k][1], t);
      rv[i][k] = fma(dx[i][k][2], dv[i][k][2], t);
      d2[i][k] = r2;
    }
  auto dist2 = [&](int i, int k) -> double { return i == 0 ? q2[k] : d2[i][k]; };
  if (FIRST) {
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int k = (i == 0 ? 1 : i + 1); k < N; k++) rho[i][k] = rsqrt(dist2(i, k));
  } else {
    double del[N][N];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int k = (i == 0 ? 1 : i + 1); k < N; k++) {
        del[i][k] = fma(dist2(i, k), rc.r2[i][k], -1.0);
        ok &= (__double2hiint(del[i][k]) & 0x7ff00000) < ((1023 - 20) << 20);  // |delta| < 2^-20, integer pipe
      }
    if (ok) {
#pragma unroll
      for (int i = 0; i < N; i++)
#pragma unroll
        for (int k = (i == 0 ? 1 : i + 1); k < N; k++)
          rho[i][k] = fma(kmul(kk, rc.r[i][k], del[i][k]), fma(0.375, del[i][k], -0.5), rc.r[i][k]);
    } else {
#pragma unroll
      for (int i = 0; i < N; i++)
#pragma unroll
        for (int k = (i == 0 ? 1 : i + 1); k < N; k++) rho[i][k] = rsqrt_call(dist2(i, k));
    }
  }
  // body 0's pairs: A_k = -m_0 s_k X_k - a_0, a_0 = sum_j m_j s_j X_j (likewise J)
  double w0[N][3], m0s[N], IA[3], IJ[3];
#pragma unroll
  for (int k = 1; k < N; k++) {
    const double rho2 = kmul(kk, rho[0][k], rho[0][k]);
    rc.r[0][k] = rho[0][k];
    rc.r2[0][k] = rho2;
    const double s3 = kmul(kk, rho2, rho[0][k]);
    const double cc = kmul(kk, -3.0, kmul(kk, rv[0][k], rho2));
    const double ms = kmul(kk, m[k], s3);
    m0s[k] = kmul(kk, m[0], s3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      w0[k][c] = fma(cc, X[k][c], V[k][c]);
      IA[c] = k == 1 ? kmul(kk, ms, X[k][c]) : fma(ms, X[k][c], IA[c]);
      IJ[c] = k == 1 ? kmul(kk, ms, w0[k][c]) : fma(ms, w0[k][c], IJ[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    A[0][c] = IA[c];
    J[0][c] = IJ[c];
  }
#pragma unroll
  for (int k = 1; k < N; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      A[k][c] = fma(-m0s[k], X[k][c], -IA[c]);
      J[k][c] = fma(-m0s[k], w0[k][c], -IJ[c]);
    }
  // pairs of bodies i, k >= 1
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) {
      const double rho2 = kmul(kk, rho[i][k], rho[i][k]);
      rc.r[i][k] = rho[i][k];
      rc.r2[i][k] = rho2;
      const double rho3 = kmul(kk, rho2, rho[i][k]);
      const double cc = kmul(kk, -3.0, kmul(kk, rv[i][k], rho2));
      const double sk = kmul(kk, m[k], rho3), si = kmul(kk, m[i], rho3);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const double w = fma(cc, dx[i][k][c], dv[i][k][c]);
        A[i][c] = fma(sk, dx[i][k][c], A[i][c]);
        J[i][c] = fma(sk, w, J[i][c]);
        A[k][c] = fma(-si, dx[i][k][c], A[k][c]);
        J[k][c] = fma(-si, w, J[k][c]);
      }
    }
}

template <int N>
__device__ __forceinline__ void spl_energy(const double (&x)[N][3], const double (&v)[N][3], const double (&m)[N],
                                           double (&out)[4]) {
  double e = 0, L0 = 0, L1 = 0, L2 = 0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    e += 0.5 * m[i] * (v[i][0] * v[i][0] + v[i][1] * v[i][1] + v[i][2] * v[i][2]);
    L0 += m[i] * (x[i][1] * v[i][2] - x[i][2] * v[i][1]);
    L1 += m[i] * (x[i][2] * v[i][0] - x[i][0] * v[i][2]);
    L2 += m[i] * (x[i][0] * v[i][1] - x[i][1] * v[i][0]);
#pragma unroll
    for (int k = i + 1; k < N; k++) {
      double d0 = x[k][0] - x[i][0], d1 = x[k][1] - x[i][1], d2 = x[k][2] - x[i][2];
      e -= m[i] * m[k] * rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
  }
  out[0] = e;
  out[1] = L0;
  out[2] = L1;
  out[3] = L2;
}

// Close-encounter test of one planet pair: |x_i - x_j| < f k_ij (q_i + q_j)/2 with
// kc = (f k_ij / 2)^2, k_ij = ((m_i + m_j)/(3 m_0))^(1/3).  The bound
// (q_i + q_j)^2 <= 2 (q_i^2 + q_j^2) rules most pairs out without a square root.
__device__ __forceinline__ bool close_encounter(const F64k &k, double d2, double kc, double q2i, double q2j) {
  double t = kadd(k, q2i, q2j);
  if (nonneg_lt(d2, kmul(k, kmul(k, 2.0, kc), t))) {  // squared distances: integer compare
    double s = sqrt(q2i) + sqrt(q2j);
    return d2 < kc * (s * s);
  }
  return false;
}

__device__ __forceinline__ double hill_kc(double ce, double mi, double mj, double m0) {
  if (!(ce > 0)) return 0.0;
  double k = cbrt((mi + mj) / (3.0 * m0));
  double f = 0.5 * ce * k;
  return f * f;
}

__device__ __forceinline__ void write_log(const StepParams &P, int gsys, double t, const double (&e)[4]) {
  int c = P.log_count[gsys];
  int slot = c % P.log_cap;
  double *rec = P.log + ((size_t)gsys * P.log_cap + slot) * 5;
  rec[0] = t;
  rec[1] = e[0];
  rec[2] = e[1];
  rec[3] = e[2];
  rec[4] = e[3];
  P.log_count[gsys] = c + 1;
}

}  // namespace swarm
