// Host-side plan: the plane-wave sphere of a k-point, its z-sticks and m1-planes, and the
// radix/twiddle plans of the warp FFT.  (Paper Sec. 3: PW basis with a kinetic cutoff;
// App. A.2.1 writes PWs as |k+G>.)
#include <cmath>
#include <cstdio>

#include "hpsi_internal.h"

namespace hpsi {

static const double kTwoPi = 6.283185307179586476925286766559;

// b_j = 2 pi (a_k x a_l) / (a_1 . (a_2 x a_3)), (j, k, l) cyclic: a_i . b_j = 2 pi delta_ij.
void reciprocal(const double a[9], double b[9]) {
  const double* a1 = a;
  const double* a2 = a + 3;
  const double* a3 = a + 6;
  double c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2], a2[0] * a3[1] - a2[1] * a3[0]};
  double c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2], a3[0] * a1[1] - a3[1] * a1[0]};
  double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
  double vol = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
  for (int i = 0; i < 3; ++i) {
    b[i] = kTwoPi * c23[i] / vol;
    b[3 + i] = kTwoPi * c31[i] / vol;
    b[6 + i] = kTwoPi * c12[i] / vol;
  }
}

// {G = m.b : |k+G|^2/2 <= ecut}, signed Miller indices in lexicographic order.
int enumerate_gsphere(const double cell[9], double ecut, const double k[3], std::vector<int32_t>& miller,
                      std::string& err) {
  if (!(ecut > 0.0) || !std::isfinite(ecut)) {
    err = "ecut must be a positive finite number";
    return HPSI_EINVAL;
  }
  double b[9];
  reciprocal(cell, b);
  double vol = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
               cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
  if (!(std::fabs(vol) > 1e-12) || !std::isfinite(vol)) {
    err = "cell is singular";
    return HPSI_EINVAL;
  }
  const double qmax = std::sqrt(2.0 * ecut);
  long lo[3], hi[3];
  double span = 1.0;
  for (int i = 0; i < 3; ++i) {
    const double* ai = cell + 3 * i;
    double kf = (k[0] * ai[0] + k[1] * ai[1] + k[2] * ai[2]) / kTwoPi;
    double r = qmax * std::sqrt(ai[0] * ai[0] + ai[1] * ai[1] + ai[2] * ai[2]) / kTwoPi;
    lo[i] = (long)std::floor(-kf - r) - 1;
    hi[i] = (long)std::ceil(-kf + r) + 1;
    span *= (double)(hi[i] - lo[i] + 1);
  }
  if (span > 2.0e8) {
    err = "cutoff too large for the cell (more than 2e8 candidate G vectors)";
    return HPSI_EINVAL;
  }
  miller.clear();
  for (long m1 = lo[0]; m1 <= hi[0]; ++m1)
    for (long m2 = lo[1]; m2 <= hi[1]; ++m2)
      for (long m3 = lo[2]; m3 <= hi[2]; ++m3) {
        double q[3];
        for (int c = 0; c < 3; ++c) q[c] = k[c] + (double)m1 * b[c] + (double)m2 * b[3 + c] + (double)m3 * b[6 + c];
        double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        if (0.5 * q2 <= ecut) {
          miller.push_back((int32_t)m1);
          miller.push_back((int32_t)m2);
          miller.push_back((int32_t)m3);
        }
      }
  return HPSI_OK;
}

bool fft_size_ok(int n) {
  if (n < 8 || n > kMaxFftN) return false;
  int r = n;
  for (int p : {2, 3, 5})
    while (r % p == 0) r /= p;
  return r == 1;
}

// Radices: as many 4s as possible, then 2, 3, 5.  Twiddles of stage s (radix R, Ns = product of
// earlier radices): w[k][r-1] = exp(-2 pi i r k / (Ns R)), k < Ns, r = 1..R-1, from host sin/cos.
void make_fft_plan(int n, FftPlan& plan, std::vector<double2>& table) {
  plan.n = n;
  plan.nstages = 0;
  int r = n;
  int rad[kMaxStages];
  int ns = 0;
  while (r % 4 == 0) { rad[ns++] = 4; r /= 4; }
  for (int p : {2, 3, 5})
    while (r % p == 0) { rad[ns++] = p; r /= p; }
  table.clear();
  int Ns = 1;
  for (int s = 0; s < ns; ++s) {
    int R = rad[s];
    plan.radix[s] = R;
    plan.twoff[s] = (int)table.size();
    for (int kk = 0; kk < Ns; ++kk)
      for (int rr = 1; rr < R; ++rr) {
        double ang = -kTwoPi * (double)(rr * kk) / (double)(Ns * R);
        table.push_back(make_double2(std::cos(ang), std::sin(ang)));
      }
    Ns *= R;
  }
  plan.nstages = ns;
  plan.tw64 = nullptr;
  plan.tw32 = nullptr;
}

static int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Sticks (distinct (m1, m2)) and planes (distinct m1) of the sphere, the kinetic diagonal.
int build_geometry(Problem& p, std::string& err) {
  const int npw = (int)(p.miller.size() / 3);
  p.npw = npw;
  p.sticks.clear();
  p.planes.clear();
  p.kin.assign(npw, 0.0);
  int mmax[3] = {0, 0, 0};
  for (int g = 0; g < npw; ++g)
    for (int c = 0; c < 3; ++c) mmax[c] = std::max(mmax[c], std::abs(p.miller[3 * g + c]));
  for (int c = 0; c < 3; ++c) {
    if (!fft_size_ok(p.n[c])) {
      err = "FFT edge " + std::to_string(p.n[c]) + " is not a 2*3*5-smooth integer in [8, 256]";
      return HPSI_EINVAL;
    }
    if (p.n[c] < 2 * mmax[c] + 1) {
      err = "FFT box too small for the sphere: n" + std::to_string(c + 1) + " = " + std::to_string(p.n[c]) +
            " < " + std::to_string(2 * mmax[c] + 1);
      return HPSI_EINVAL;
    }
  }
  int prev1 = INT32_MIN, prev2 = INT32_MIN;
  for (int g = 0; g < npw; ++g) {
    int m1 = p.miller[3 * g], m2 = p.miller[3 * g + 1], m3 = p.miller[3 * g + 2];
    if (m1 != prev1) {
      PlaneDev pl;
      pl.s0 = (int)p.sticks.size();
      pl.ns = 0;
      pl.ix = pmod(m1, p.n[0]);
      pl.g0 = g;
      p.planes.push_back(pl);
      prev1 = m1;
      prev2 = INT32_MIN;
    }
    if (m2 != prev2) {
      StickDev st;
      st.g0 = g;
      st.len = 0;
      st.z0 = pmod(m3, p.n[2]);
      st.iy = pmod(m2, p.n[1]);
      p.sticks.push_back(st);
      p.planes.back().ns++;
      prev2 = m2;
    }
    p.sticks.back().len++;
    double q[3];
    for (int c = 0; c < 3; ++c)
      q[c] = p.k[c] + (double)m1 * p.recip[c] + (double)m2 * p.recip[3 + c] + (double)m3 * p.recip[6 + c];
    p.kin[g] = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  }
  p.nst = (int)p.sticks.size();
  p.npl = (int)p.planes.size();
  p.ns_max = 0;
  for (auto& pl : p.planes) p.ns_max = std::max(p.ns_max, pl.ns);
  return HPSI_OK;
}

}  // namespace hpsi
