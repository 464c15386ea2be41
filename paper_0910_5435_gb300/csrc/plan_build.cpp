// plan_build.cpp -- host precomputation of the butterfly factor streams.
//
//   gl_nodes              Section 2, eq. thetas (Gauss-Legendre nodes/weights)
//   ColumnStream          Section 2.3 eqs. c_rec, d_rec, recurrence0, recurrence
//                         (x^2 recurrence) with exponent tracking (Section 4)
//   interp_decomp         Section 2.1, Remark QR_algorithm (pivoted-QR ID)
//   factor_unit           Section 2.2 eqs. 1-6, top, bottom (butterfly) built in
//                         the depth-first order of Section 3
//   emit_streams          record and value encoding of sht_stream.h (scheduled
//                         work items; staged streams for single blocks)
//
// All arithmetic is float64; nothing here runs on the hot path.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <thread>

#include "plan_host.h"

namespace sht {

namespace {

// ------------------------------------------------------------ GL nodes
//
// Only +, -, *, / and sqrt (all correctly rounded in IEEE arithmetic) are
// used, and the library is compiled without floating-point contraction, so
// the nodes, weights and sines are the same bits on every host.

// sin a and cos a for 0 <= a <= pi/2: the Taylor series at a/8 (12 terms,
// far below rounding there), then three double-angle steps.  Accurate to a
// few units in the last place, which is ample for starting Newton's method.
void series_sincos(double a, double& s, double& c) {
  const double h = a / 8.0, h2 = h * h;
  double ts = h, tc = 1.0;
  s = h;
  c = 1.0;
  for (int k = 1; k <= 12; ++k) {
    ts = -ts * h2 / ((2.0 * k) * (2.0 * k + 1.0));
    tc = -tc * h2 / ((2.0 * k - 1.0) * (2.0 * k));
    s += ts;
    c += tc;
  }
  for (int r = 0; r < 3; ++r) {
    const double s2 = 2.0 * s * c;
    c = (c - s) * (c + s);
    s = s2;
  }
}

// P_n(x) and P_{n-1}(x) for the unnormalized Legendre polynomials, from
// (j + 1) P_{j+1} = (2j + 1) x P_j - j P_{j-1}.  The coefficients are exact
// integers, so the only rounding is in the arithmetic itself; the normalized
// form's rounded square-root coefficients cost an order of magnitude in the
// weights near the poles.
void legendre_pn(int n, double x, double& pn, double& pn1) {
  double p0 = 1.0, p1 = x;
  for (int j = 1; j < n; ++j) {
    const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pn1 = p0;
}

}  // namespace

void gl_nodes(int npts, std::vector<double>& x, std::vector<double>& w, std::vector<double>& sin_pos,
              int threads) {
  if (npts < 2 || (npts & 1)) throw std::invalid_argument("gl_nodes: npts must be even");
  const int n = npts, half = n / 2;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  sin_pos.assign(half, 0.0);
  const double pi = 3.14159265358979323846;
  // each node is computed on its own, so the thread count cannot change a bit
  auto one_node = [&](int k) {
    // start: theta ~ phi + cot(phi) / (8 (n + 1/2)^2), phi = pi (k - 1/4) / (n + 1/2)
    const double phi = pi * (k - 0.25) / (n + 0.5);
    double sp, cp, sth, xk;
    series_sincos(phi, sp, cp);
    series_sincos(phi + cp / (sp * 8.0 * (n + 0.5) * (n + 0.5)), sth, xk);
    // Newton on P_n in x, with P_n' = n (P_{n-1} - x P_n) / (1 - x^2); once a
    // step is below 8 units in the last place of x, one more step and stop
    double p, pm;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(n, xk, p, pm);
      const double step = p / (n * (pm - xk * p) / ((1.0 - xk) * (1.0 + xk)));
      xk -= step;
      if (std::fabs(step) <= 0x1p-50 * xk) {
        legendre_pn(n, xk, p, pm);
        xk -= p / (n * (pm - xk * p) / ((1.0 - xk) * (1.0 + xk)));
        break;
      }
    }
    // The root r = xk + d lies within rounding of xk: the weight
    // w = 2 / ((1 - r^2) P_n'(r)^2) and sin theta = sqrt(1 - r^2) are taken
    // at r, with P_n'(r) = P_n'(xk) + P_n''(xk) d from Legendre's equation
    // (1 - x^2) P'' = 2 x P' - n (n + 1) P.
    legendre_pn(n, xk, p, pm);
    const double omx2 = (1.0 - xk) * (1.0 + xk);
    const double dp = n * (pm - xk * p) / omx2;
    const double d = -p / dp;
    const double d2p = (2.0 * xk * dp - n * (n + 1.0) * p) / omx2;
    const double dpr = dp + d2p * d;
    const double omr2 = omx2 - 2.0 * xk * d - d * d;
    const double wk = 2.0 / (omr2 * dpr * dpr);
    // k = 1 is the largest node; positive nodes sit at indices half..n-1 ascending
    x[n - k] = xk;
    x[k - 1] = -xk;
    w[n - k] = wk;
    w[k - 1] = wk;
    sin_pos[half - k] = std::sqrt(omr2);
  };
  constexpr int kChunk = 16;
  const int nchunks = (half + kChunk - 1) / kChunk;
  const int avail = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  const int nt = std::max(1, std::min({avail, nchunks, 64}));
  std::atomic<int> next(0);
  auto worker = [&]() {
    for (int c; (c = next.fetch_add(1)) < nchunks;)
      for (int k = 1 + c * kChunk; k <= std::min(half, (c + 1) * kChunk); ++k) one_node(k);
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
}

// ------------------------------------------------------- column stream

namespace {
inline void renorm(double& v, int& e) {
  if (v == 0.0) return;
  int t;
  v = std::frexp(v, &t);
  e += t;
}
}  // namespace

ColumnStream::ColumnStream(const PlanHost& P, int m, int p, int rows, int row0)
    : m_(m), p_(p), rows_(rows), j_(0) {
  const int l = P.l;
  x2_.resize(rows);
  sq2w_.resize(rows);
  a_.assign(rows, 0.0);
  b_.resize(rows);
  e_.resize(rows);
  // c_m = (1/sqrt 2) prod_{j=1}^m sqrt((2j+1)/(2j)): P-bar^m_m(x) = c_m (1-x^2)^{m/2}
  // (eq. association with d^m P_m / dx^m = (2m)! / (2^m m!))
  double cm = 1.0 / std::sqrt(2.0);
  int ecm = 0;
  for (int j = 1; j <= m; ++j) {
    cm *= std::sqrt((2.0 * j + 1.0) / (2.0 * j));
    renorm(cm, ecm);
  }
  const bool custom = !P.row_x.empty();
  for (int i = 0; i < rows; ++i) {
    const int g = row0 + i;
    const double xi = custom ? P.row_x[g] : P.x[l + g];
    const double s = custom ? P.row_sin[g] : P.sin_pos[g];
    x2_[i] = xi * xi;
    sq2w_[i] = custom ? P.row_sqw[g] : std::sqrt(2.0 * P.w[l + g]);
    // s^m by binary powering with tracked exponents
    int eb;
    double base = std::frexp(s, &eb);
    double res = 1.0;
    int er = 0;
    for (int q = m; q; q >>= 1) {
      if (q & 1) {
        res *= base;
        er += eb;
        renorm(res, er);
      }
      base *= base;
      eb *= 2;
      renorm(base, eb);
    }
    double v = res * cm;
    int ev = er + ecm;
    if (p == 1) v *= std::sqrt(2.0 * m + 3.0) * xi;  // P-bar^m_{m+1} = sqrt(2m+3) x P-bar^m_m
    renorm(v, ev);
    b_[i] = v;
    e_[i] = ev;
  }
}

void ColumnStream::next(double* col) {
  const int k = m_ + p_ + 2 * j_;
  // b 2^e: one product with an exact power of two where 2^e is a normal
  // number (the same correctly rounded value as ldexp), ldexp otherwise
  for (int i = 0; i < rows_; ++i) {
    const int e = e_[i];
    double s;
    if (e >= -1022 && e <= 1023) {
      const uint64_t bits = (uint64_t)(e + 1023) << 52;
      double p2;
      std::memcpy(&p2, &bits, 8);
      s = b_[i] * p2;
    } else {
      s = std::ldexp(b_[i], e);
    }
    col[i] = sq2w_[i] * s;
  }
  // advance P-bar_k -> P-bar_{k+2}: x^2 P_k = c_{k-2} P_{k-2} + d_k P_k + c_k P_{k+2}
  const double ck = rec_c(k, m_), dk = rec_d(k, m_);
  const double ckm2 = (j_ > 0) ? rec_c(k - 2, m_) : 0.0;  // eq. recurrence0 for j = 0
  const double inv_ck = 1.0 / ck;
  for (int i = 0; i < rows_; ++i) {
    const double nb = ((x2_[i] - dk) * b_[i] - ckm2 * a_[i]) * inv_ck;
    a_[i] = b_[i];
    b_[i] = nb;
    const double big = std::max(std::fabs(a_[i]), std::fabs(b_[i]));
    if (big > 0x1p400 || (big < 0x1p-400 && big > 0.0)) {
      const int t = std::ilogb(big);
      a_[i] = std::ldexp(a_[i], -t);
      b_[i] = std::ldexp(b_[i], -t);
      e_[i] += t;
    }
  }
  ++j_;
}

// ------------------------------------------------------------------ ID

namespace {
// sum_{r < n} a[r] b[r] with four partial sums (independent add chains, so
// the loop is not bound by the latency of one chain of additions)
inline double dot4(const double* a, const double* b, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int r = 0;
  for (; r + 4 <= n; r += 4) {
    s0 += a[r] * b[r];
    s1 += a[r + 1] * b[r + 1];
    s2 += a[r + 2] * b[r + 2];
    s3 += a[r + 3] * b[r + 3];
  }
  for (; r < n; ++r) s0 += a[r] * b[r];
  return (s0 + s1) + (s2 + s3);
}
// y[r] -= d x[r], r < n (y and x are different columns)
inline void axpy_neg(double* __restrict y, const double* __restrict x, double d, int n) {
  for (int r = 0; r < n; ++r) y[r] -= d * x[r];
}
}  // namespace

int interp_decomp(double* A, int h, int w, double eps, std::vector<int>& perm, std::vector<double>& T, int* swaps) {
  perm.resize(w);
  std::iota(perm.begin(), perm.end(), 0);
  T.clear();
  if (swaps) *swaps = 0;
  if (w == 0) return 0;
  const std::vector<double> orig(A, A + (size_t)h * w);  // for refactoring after exchanges
  std::vector<double> nrm(w), ref(w);
  for (int j = 0; j < w; ++j) {
    const double* c = A + (size_t)j * h;
    nrm[j] = ref[j] = dot4(c, c, h);
  }
  const double eps2 = eps * eps;
  const int kmax = std::min(h, w);
  int k = 0;
  auto exact_norm = [&](int j, int i0) {
    const double* c = A + (size_t)j * h + i0;
    return dot4(c, c, h - i0);
  };
  // Householder reflector for A[i:h, i], applied to columns i+1..w-1
  auto reflect = [&](int i) {
    double* ci = A + (size_t)i * h;
    const double alpha = ci[i];
    const double sigma = dot4(ci + i + 1, ci + i + 1, h - i - 1);
    double tau = 0.0;
    if (sigma != 0.0 || alpha < 0.0) {
      const double nx = std::sqrt(alpha * alpha + sigma);
      const double beta = (alpha <= 0.0) ? nx : -nx;
      tau = (beta - alpha) / beta;
      const double sc = 1.0 / (alpha - beta);
      for (int r = i + 1; r < h; ++r) ci[r] *= sc;
      ci[i] = beta;
    }
    if (tau != 0.0) {
      for (int j = i + 1; j < w; ++j) {
        double* cj = A + (size_t)j * h;
        double dot = cj[i] + dot4(ci + i + 1, cj + i + 1, h - i - 1);
        dot *= tau;
        cj[i] -= dot;
        axpy_neg(cj + i + 1, ci + i + 1, dot, h - i - 1);
      }
    }
  };
  for (int i = 0; i < kmax; ++i) {
    int p = i;
    for (int j = i + 1; j < w; ++j)
      if (nrm[j] > nrm[p]) p = j;  // ties: lowest index
    nrm[p] = exact_norm(p, i);
    if (nrm[p] <= eps2) {
      // the downdated norms may have drifted: recompute all before stopping
      for (int j = i; j < w; ++j) nrm[j] = ref[j] = exact_norm(j, i);
      p = i;
      for (int j = i + 1; j < w; ++j)
        if (nrm[j] > nrm[p]) p = j;
      if (nrm[p] <= eps2) break;
    }
    if (p != i) {
      std::swap_ranges(A + (size_t)i * h, A + (size_t)i * h + h, A + (size_t)p * h);
      std::swap(nrm[i], nrm[p]);
      std::swap(ref[i], ref[p]);
      std::swap(perm[i], perm[p]);
    }
    reflect(i);
    for (int j = i + 1; j < w; ++j) {
      const double rij = A[(size_t)j * h + i];
      nrm[j] -= rij * rij;
      if (nrm[j] < 1e-4 * ref[j]) nrm[j] = ref[j] = exact_norm(j, i + 1);
    }
    k = i + 1;
  }
  // T = R11^{-1} R12 by back substitution, column by column
  const int nred = w - k;
  auto solve = [&]() {
    T.assign((size_t)k * nred, 0.0);
    for (int s = 0; s < nred; ++s) {
      const double* rc = A + (size_t)(k + s) * h;
      double* tc = T.data() + (size_t)s * k;
      for (int t = k - 1; t >= 0; --t) {
        double v = rc[t];
        for (int t2 = t + 1; t2 < k; ++t2) v -= A[(size_t)t2 * h + t] * tc[t2];
        tc[t] = v / A[(size_t)t * h + t];
      }
    }
  };
  solve();
  // Strong rank-revealing step (Remark QR_algorithm: interpolation
  // coefficients at most 2).  While some |T(t, s)| > 2, exchange skeleton
  // column t with redundant column s and refactor the columns in the new
  // order without pivoting.  An exchange multiplies |det R11| by at least
  // |T(t, s)| > 2, so the loop ends; it is capped at 2k exchanges.
  int nswap = 0;
  while (k > 0 && nred > 0 && nswap < 2 * k) {
    size_t best = 0;
    for (size_t x = 1; x < T.size(); ++x)
      if (std::fabs(T[x]) > std::fabs(T[best])) best = x;
    if (!(std::fabs(T[best]) > 2.0)) break;
    const int s = (int)(best / k), t = (int)(best % k);
    std::swap(perm[t], perm[k + s]);
    for (int j = 0; j < w; ++j)
      std::copy(orig.begin() + (size_t)perm[j] * h, orig.begin() + (size_t)(perm[j] + 1) * h, A + (size_t)j * h);
    for (int i = 0; i < k; ++i) reflect(i);
    solve();
    ++nswap;
  }
  if (swaps) *swaps = nswap;
  // redundant columns in ascending order (T columns follow)
  std::vector<int> ord(nred);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return perm[k + a] < perm[k + b]; });
  std::vector<int> red(nred);
  std::vector<double> T2(T.size());
  for (int s = 0; s < nred; ++s) {
    red[s] = perm[k + ord[s]];
    std::copy(T.begin() + (size_t)ord[s] * k, T.begin() + (size_t)(ord[s] + 1) * k, T2.begin() + (size_t)s * k);
  }
  std::copy(red.begin(), red.end(), perm.begin() + k);
  T.swap(T2);
  return k;
}

// ------------------------------------------------------- butterflies

namespace {

struct BandData {
  int r0 = 0, r1 = 0, k = 0;
  std::vector<double> Ask;  // (r1 - r0) x k, column-major: the skeleton columns
};
struct Group {
  int level = 0, g = 0;
  std::vector<BandData> bands;
};

long long group_words(const std::vector<Group>& st) {
  long long s = 0;
  for (const auto& g : st)
    for (const auto& b : g.bands) s += (long long)b.Ask.size();
  return s;
}

UnitFact factor_unit(const PlanHost& P, int m, int p, double eps) {
  UnitFact U;
  U.m = m;
  U.p = p;
  const int l = P.l, L = 2 * l;
  const int n = P.unit_cols > 0 ? P.unit_cols : std::max(0, (L - m - p + 1) / 2);
  U.n = n;
  if (n == 0) return U;

  // trimming: rows whose weighted norm is below trim/sqrt(l) (a suffix) are
  // dropped.  Only the last row that reaches the threshold matters, so rows
  // are tried from the pole down, 64 at a time, and a chunk's columns stop
  // once every row in it has reached the threshold (a sum only grows): the
  // same decision as summing every row over every column.
  int rows = l;
  if (P.trim_eps > 0.0) {
    const double thr = P.trim_eps / std::sqrt((double)l);
    const double thr2 = thr * thr;
    constexpr int kChunk = 64;
    std::vector<double> col(kChunk), nr(kChunk);
    rows = 0;
    for (int top = l; top > 0 && rows == 0; top -= kChunk) {
      const int r0 = std::max(0, top - kChunk), nrows = top - r0;
      ColumnStream cs(P, m, p, nrows, r0);
      std::fill(nr.begin(), nr.end(), 0.0);
      int reached = 0;
      for (int j = 0; j < n && reached < nrows; ++j) {
        cs.next(col.data());
        reached = 0;
        for (int i = 0; i < nrows; ++i) {
          if (nr[i] < thr2) nr[i] += col[i] * col[i];
          reached += nr[i] >= thr2;
        }
      }
      for (int i = nrows - 1; i >= 0 && rows == 0; --i)
        if (nr[i] >= thr2) rows = r0 + i + 1;
    }
  }
  U.rows = rows;
  if (rows == 0) return U;

  const int C = P.leaf_cols;
  int lam = 0;
  while ((n >> lam) > C) ++lam;  // 2^lam leaves of width <= ~C
  if (n > C && (n + (1 << lam) - 1) / (1 << lam) > C) ++lam;
  while (lam > 0 && (rows >> lam) < P.min_band_rows) --lam;
  const int nleaves = 1 << lam;

  // depth-first construction (Section 3): each full-height leaf is built only
  // after everything to its left has been merged as far as possible.
  ColumnStream cs(P, m, p, rows);
  std::vector<Group> stack;
  std::vector<int> perm;
  std::vector<double> T;
  long long peak = 0;
  for (int g = 0; g < nleaves; ++g) {
    const int c0 = (int)((long long)g * n / nleaves), c1 = (int)((long long)(g + 1) * n / nleaves);
    const int wd = c1 - c0;
    std::vector<double> leaf((size_t)rows * wd);
    for (int j = 0; j < wd; ++j) cs.next(leaf.data() + (size_t)j * rows);
    std::vector<double> work(leaf);
    int sw = 0;
    const int k = interp_decomp(work.data(), rows, wd, eps, perm, T, &sw);
    U.swaps += sw;
    IdBlock b;
    b.level = 1;
    b.band = 0;
    b.group = g;
    b.r0 = 0;
    b.r1 = rows;
    b.in_off = c0;
    b.nin = wd;
    b.k = k;
    b.skel.assign(perm.begin(), perm.begin() + k);
    b.red.assign(perm.begin() + k, perm.end());
    b.T = T;
    U.blocks.push_back(std::move(b));
    Group grp;
    grp.level = 1;
    grp.g = g;
    BandData bd;
    bd.r0 = 0;
    bd.r1 = rows;
    bd.k = k;
    bd.Ask.resize((size_t)rows * k);
    for (int t = 0; t < k; ++t)
      std::copy(leaf.begin() + (size_t)perm[t] * rows, leaf.begin() + (size_t)(perm[t] + 1) * rows,
                bd.Ask.begin() + (size_t)t * rows);
    grp.bands.push_back(std::move(bd));
    stack.push_back(std::move(grp));
    peak = std::max(peak, group_words(stack) + (long long)leaf.size() * 2);

    while (stack.size() >= 2 && stack[stack.size() - 1].level == stack[stack.size() - 2].level) {
      Group R = std::move(stack.back());
      stack.pop_back();
      Group Lg = std::move(stack.back());
      stack.pop_back();
      const int j = Lg.level;
      Group ng;
      ng.level = j + 1;
      ng.g = Lg.g / 2;
      ng.bands.resize(Lg.bands.size() * 2);
      for (size_t beta = 0; beta < Lg.bands.size(); ++beta) {
        const BandData& BL = Lg.bands[beta];
        const BandData& BR = R.bands[beta];
        const int h = BL.r1 - BL.r0, mid = BL.r0 + h / 2;
        const int kin = BL.k + BR.k;
        for (int half = 0; half < 2; ++half) {
          const int rr0 = half ? mid : BL.r0, rr1 = half ? BL.r1 : mid, hh = rr1 - rr0;
          std::vector<double> Z((size_t)hh * kin);
          for (int t = 0; t < BL.k; ++t)
            std::copy(BL.Ask.begin() + (size_t)t * h + (rr0 - BL.r0), BL.Ask.begin() + (size_t)t * h + (rr1 - BL.r0),
                      Z.begin() + (size_t)t * hh);
          for (int t = 0; t < BR.k; ++t)
            std::copy(BR.Ask.begin() + (size_t)t * h + (rr0 - BL.r0), BR.Ask.begin() + (size_t)t * h + (rr1 - BL.r0),
                      Z.begin() + (size_t)(BL.k + t) * hh);
          std::vector<double> Zw(Z);
          int sw = 0;
          const int k = interp_decomp(Zw.data(), hh, kin, eps, perm, T, &sw);
          U.swaps += sw;
          IdBlock b;
          b.level = j + 1;
          b.band = (int)(2 * beta + half);
          b.group = ng.g;
          b.r0 = rr0;
          b.r1 = rr1;
          b.nin = kin;
          b.k = k;
          b.skel.assign(perm.begin(), perm.begin() + k);
          b.red.assign(perm.begin() + k, perm.end());
          b.T = T;
          U.blocks.push_back(std::move(b));
          BandData nb;
          nb.r0 = rr0;
          nb.r1 = rr1;
          nb.k = k;
          nb.Ask.resize((size_t)hh * k);
          for (int t = 0; t < k; ++t)
            std::copy(Z.begin() + (size_t)perm[t] * hh, Z.begin() + (size_t)(perm[t] + 1) * hh,
                      nb.Ask.begin() + (size_t)t * hh);
          ng.bands[2 * beta + half] = std::move(nb);
        }
      }
      stack.push_back(std::move(ng));
      peak = std::max(peak, group_words(stack));
    }
  }
  U.peak_words = peak;
  U.levels = lam;
  // top level: one group, 2^lam bands whose stored skeleton columns are the final blocks
  std::vector<FinalBlock> top;
  for (size_t beta = 0; beta < stack.back().bands.size(); ++beta) {
    BandData& bd = stack.back().bands[beta];
    FinalBlock f;
    f.band = (int)beta;
    f.r0 = bd.r0;
    f.r1 = bd.r1;
    f.k = bd.k;
    f.S = std::move(bd.Ask);  // column-major h x k == S[t * h + i]
    top.push_back(std::move(f));
  }
  finish_unit(P, U, std::move(top));
  return U;
}

}  // namespace

void finish_unit(const PlanHost& P, UnitFact& U, std::vector<FinalBlock>&& top) {
  const int lam = U.levels, rows = U.rows, n = U.n, m = U.m, p = U.p;
  // layouts: level j holds its blocks band-major, group-minor
  U.width.assign(lam + 2, 0);
  std::vector<std::vector<int>> at(lam + 2);
  for (int bi = 0; bi < (int)U.blocks.size(); ++bi) at[U.blocks[bi].level].push_back(bi);
  for (int j = 1; j <= lam + 1; ++j) {
    auto& v = at[j];
    std::sort(v.begin(), v.end(), [&](int a, int b) {
      const IdBlock &A = U.blocks[a], &B = U.blocks[b];
      return A.band != B.band ? A.band < B.band : A.group < B.group;
    });
    int off = 0;
    for (int bi : v) {
      U.blocks[bi].out_off = off;
      off += U.blocks[bi].k;
    }
    U.width[j] = off;
  }
  // input offsets of merge blocks: z = [y(L); y(R)] of the parent band, groups 2g and 2g+1
  for (int j = 2; j <= lam + 1; ++j) {
    for (int bi : at[j]) {
      IdBlock& B = U.blocks[bi];
      const int pb = B.band / 2;
      int found = -1;
      for (int ci : at[j - 1])
        if (U.blocks[ci].band == pb && U.blocks[ci].group == 2 * B.group) found = ci;
      if (found < 0) throw std::logic_error("butterfly layout: missing left child");
      B.in_off = U.blocks[found].out_off;
    }
  }
  for (FinalBlock& f : top) {
    for (int bi : at[lam + 1])
      if (U.blocks[bi].band == f.band) f.in_off = U.blocks[bi].out_off;
    U.finals.push_back(std::move(f));
  }
  for (const auto& b : U.blocks) {
    U.values += (long long)b.k * (b.nin - b.k);
    U.idx += b.nin;
  }
  for (const auto& f : U.finals) U.values += (long long)f.k * (f.r1 - f.r0);

  // a dense block is cheaper when compression does not pay
  const double bfly_bytes = 8.0 * U.values + 2.0 * U.idx + 48.0 * (U.blocks.size() + U.finals.size());
  const double dense_bytes = 8.0 * rows * (double)n;
  if (dense_bytes <= bfly_bytes) {
    U.direct = true;
    U.blocks.clear();
    U.finals.clear();
    U.width.clear();
    U.levels = 0;
    U.values = (long long)rows * n;
    U.idx = 0;
    U.D.resize((size_t)rows * n);
    ColumnStream cs2(P, m, p, rows);
    for (int j = 0; j < n; ++j) cs2.next(U.D.data() + (size_t)j * rows);
  }
  U.cost = std::min(bfly_bytes, dense_bytes);
}

UnitFact factor_single_unit(const PlanHost& P, int m, int p, double eps) { return factor_unit(P, m, p, eps); }

long long depth_first_peak(const UnitFact& U) {
  const int lam = U.levels, nleaves = 1 << lam;
  // words kept by each group (level j, group g), and the leaves' widths
  std::vector<std::vector<long long>> words(lam + 2);
  for (int j = 1; j <= lam + 1; ++j) words[j].assign(std::max(1, nleaves >> (j - 1)), 0);
  std::vector<long long> width(nleaves, 0);
  for (const IdBlock& b : U.blocks) {
    if (b.level < 1 || b.level > lam + 1 || b.group < 0 || b.group >= (int)words[b.level].size())
      throw std::logic_error("butterfly layout: block outside its level");
    words[b.level][b.group] += (long long)(b.r1 - b.r0) * b.k;
    if (b.level == 1) width[b.group] = b.nin;
  }
  long long total = 0, peak = 0;
  std::vector<std::pair<int, int>> stack;  // (level, group)
  for (int g = 0; g < nleaves; ++g) {
    stack.push_back({1, g});
    total += words[1][g];
    peak = std::max(peak, total + 2LL * U.rows * width[g]);
    while (stack.size() >= 2 && stack[stack.size() - 1].first == stack[stack.size() - 2].first) {
      const int j = stack.back().first, gr = stack.back().second;
      stack.pop_back();
      stack.pop_back();
      total -= words[j][gr] + words[j][gr - 1];
      total += words[j + 1][gr / 2];
      stack.push_back({j + 1, gr / 2});
      peak = std::max(peak, total);
    }
  }
  return peak;
}

void build_factorizations(PlanHost& P, bool fp32) {
  const int l = P.l, L = 2 * l;
  const double eps = fp32 ? P.eps_fp32 : P.eps_id;
  std::vector<UnitFact>& out = fp32 ? P.fact32 : P.fact64;
  out.assign((size_t)L * 2, UnitFact());
  std::vector<int> order(L * 2);
  std::iota(order.begin(), order.end(), 0);
  // biggest first (n_{m,p} ~ (2l - m)/2)
  std::sort(order.begin(), order.end(), [](int a, int b) { return (a / 2) < (b / 2); });
  std::atomic<int> next(0);
  int nt = P.num_threads > 0 ? P.num_threads : (int)std::thread::hardware_concurrency();
  nt = std::max(1, std::min(nt, 256));
  std::vector<std::string> errors(nt);
  auto worker = [&](int tid) {
    try {
      for (;;) {
        const int q = next.fetch_add(1);
        if (q >= (int)order.size()) break;
        const int u = order[q];
        out[u] = factor_unit(P, u / 2, u % 2, eps);
      }
    } catch (const std::exception& e) {
      errors[tid] = e.what();
      next.store((int)order.size());
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker, t);
  worker(0);
  for (auto& t : th) t.join();
  for (auto& e : errors)
    if (!e.empty()) throw std::runtime_error(e);
}

// --------------------------------------------------------------- pages

namespace {

inline size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }

// One op of a work item before scheduling: its header (bytes, npred, idx16
// and vref are set when the item is encoded), its index lists, and the item
// op numbers it must wait for.
struct OpRec {
  OpHdr h;
  std::vector<uint16_t> idx;
  std::vector<int> preds;
  bool planted = false;  // waits for itself (failure-detection tests)
  double cost = 0;       // scheduling estimate
  int stage = 0;         // emission stage (a butterfly level, a gather, ...)
};

// value encodings per precision: 0 = FP64 (double), 1 = FP32 (float), 2 = SPLIT32 (float hi, float lo)
inline size_t value_size(int prec) { return prec == 1 ? 4 : 8; }
inline void put_value(uint8_t* dst, int prec, size_t i, double v) {
  if (prec == 0) {
    reinterpret_cast<double*>(dst)[i] = v;
  } else if (prec == 1) {
    reinterpret_cast<float*>(dst)[i] = (float)v;
  } else {
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    reinterpret_cast<float*>(dst)[2 * i] = hi;
    reinterpret_cast<float*>(dst)[2 * i + 1] = lo;
  }
}

// Dependency tracking for the op stream of one work item.  Every op lists
// its predecessors explicitly: the last writer of every shared-memory
// position or node row it reads or writes (RAW, WAW) and every reader of a
// position it overwrites since that position was last written (WAR).  Ops
// with no predecessor wait for nothing inside the item (the kernel's barrier
// at the end of every item orders it after the items before); so blocks of
// one butterfly level, and the tail of one order with the head of the next
// order of the same item, run concurrently.
struct Tracker {
  std::vector<int> last_w[kNumVecs];
  std::vector<std::vector<int>> readers[kNumVecs];
  std::unordered_map<long long, int> g_last_w;  // (m, node row) of G
  int join = -1;
  void reset(int positions) {
    for (int b = 0; b < kNumVecs; ++b) {
      last_w[b].assign(positions, -1);
      readers[b].assign(positions, {});
    }
    g_last_w.clear();
    join = -1;
  }
};

// Writes ops; numbers them within the item and attaches their predecessors.
struct Emitter {
  int prec;
  size_t vs;
  Tracker* T = nullptr;
  std::vector<uint8_t>* values = nullptr;  // value region of the item
  std::vector<OpRec> ops;                  // the item's ops, in emission (topological) order
  bool plant_unmet = false;  // next compute op waits for itself (failure-detection tests)
  int slot_values = kDefaultSlotValues;  // cap on an op's values
  size_t chunk = kDefaultChunkBytes;     // a record must fit one chunk
  int next_op = 0;    // number of the next op within the item
  int positions = 0;
  int l = 0;
  // Shared-vector placement: the ops of one parity block address its vector
  // positions from `base`, chosen by place() so that consecutive blocks of a
  // work item occupy disjoint ranges whenever they fit in `pool` positions;
  // the tracker then finds no conflict between them and they run
  // concurrently (the two parities of an order, the tail of one order with
  // the head of the next).
  int base = 0;
  int cursor = 0;
  int pool = 0;
  // Stage counter: emit_unit starts a new stage before each set of mutually
  // independent ops (a gather, one butterfly level, the final blocks, ...);
  // level-by-level schedules launch each stage on its own.
  int stage = 0;
  // Vector positions are 16 bits in io / oo.  A wide emitter (single-block
  // streams, whose ops address no order) keeps the bits above in a1: io's
  // in its low half, oo's in its high half.
  bool wide = false;
  explicit Emitter(int p) : prec(p), vs(value_size(p)) {}

  void set_io_oo(OpHdr& h, long long io, long long oo) const {
    if (io < 0 || oo < 0 || (!wide && (io > 0xFFFF || oo > 0xFFFF)) || io >= (1LL << 20) || oo >= (1LL << 20))
      throw std::runtime_error("vector position out of range");
    h.io = (uint16_t)(io & 0xFFFF);
    h.oo = (uint16_t)(oo & 0xFFFF);
    if (wide) h.a1 = (uint32_t)((io >> 16) | ((oo >> 16) << 16));
  }
  long long full_io(const OpHdr& h) const { return h.io + (wide ? (long long)(h.a1 & 0xFFFF) << 16 : 0); }
  long long full_oo(const OpHdr& h) const { return h.oo + (wide ? (long long)(h.a1 >> 16) << 16 : 0); }

  // Chooses the base of a block using `width` positions of each vector.
  void place(int width) {
    if (cursor + width > pool) cursor = 0;
    base = cursor;
    cursor += width;
  }

  OpHdr hdr(uint8_t kind, uint8_t flags = 0) {
    OpHdr h;
    std::memset(&h, 0, sizeof(h));
    h.kind = kind;
    h.flags = flags;
    return h;
  }
  // Whether an op with nidx index entries and nval values is allowed: its
  // record (with room for a predecessor per warp and the planted one) fits a
  // chunk and its value block fits one warp's staging slot.
  bool fits(size_t nidx, size_t nval) const {
    return sizeof(OpHdr) + pad16(2 * (nidx + kMaxWarps + 1)) <= chunk && nval <= (size_t)slot_values;
  }

  // Reads and writes of one op, as keys: (vec << 20 | pos) for shared
  // vectors, (1 << 40 | m << 20 | row) for node rows of G.
  void access(const OpHdr& h, const std::vector<uint16_t>& idx, std::vector<long long>& R,
              std::vector<long long>& Wr) const {
    auto vkey = [](int b, long long pos) { return ((long long)b << 20) | pos; };
    auto gkey = [](int m, int row) { return (1LL << 40) | ((long long)m << 20) | row; };
    const int M = h.M, K = h.K;
    const int cbase = h.a0 >> 1;  // GATHER / SCATTER / FOLD: vector base
    const long long io = full_io(h), oo = full_oo(h);
    const uint32_t m = wide ? 0u : h.a1;  // a wide stream's ops address no order
    switch (h.kind) {
      case OP_GATHER:
      case OP_FOLD:
        for (int j = 0; j < M; ++j) Wr.push_back(vkey(h.out_buf, cbase + oo + j));
        break;
      case OP_CLEAR:
        for (int j = 0; j < M; ++j) Wr.push_back(vkey(h.out_buf, oo + j));
        break;
      case OP_SCATTER:
        for (int j = 0; j < M; ++j) R.push_back(vkey(h.in_buf, cbase + io + j));
        break;
      case OP_GZERO:
        for (int j = 0; j < M; ++j) Wr.push_back(gkey(m, l + oo + j)), Wr.push_back(gkey(m, l - 1 - oo - j));
        break;
      case OP_SYN_INTERP:
        for (int s = 0; s < K + M; ++s) R.push_back(vkey(h.in_buf, io + idx[s]));
        for (int o = 0; o < M; ++o) Wr.push_back(vkey(h.out_buf, oo + o));
        break;
      case OP_DENSE:
        for (int s = 0; s < K; ++s) R.push_back(vkey(h.in_buf, io + s));
        for (int o = 0; o < M; ++o) Wr.push_back(vkey(h.out_buf, oo + o));
        break;
      case OP_DENSE_G:
        for (int s = 0; s < K; ++s) R.push_back(vkey(h.in_buf, io + s));
        for (int o = 0; o < M; ++o) {
          Wr.push_back(gkey(m, l + oo + o));
          Wr.push_back(gkey(m, l - 1 - oo - o));
        }
        if (h.flags & F_ACCUM) R.insert(R.end(), Wr.begin(), Wr.end());
        break;
      case OP_ANA_INTERP: {
        for (int s = 0; s < K; ++s) R.push_back(vkey(h.in_buf, io + s));
        for (int o = 0; o < M; ++o) Wr.push_back(vkey(h.out_buf, oo + idx[o]));
        if (h.flags & F_SKEL)
          for (int t = 0; t < h.nskel; ++t) Wr.push_back(vkey(h.out_buf, oo + idx[M + t]));
        if (h.flags & F_ACCUM) R.insert(R.end(), Wr.begin(), Wr.end());
        break;
      }
      default:
        break;
    }
  }

  std::vector<int> preds_of(const std::vector<long long>& R, const std::vector<long long>& Wr) {
    std::vector<int> p;
    auto lw = [&](long long key) -> int {
      if (key >> 40) {
        auto it = T->g_last_w.find(key);
        return it == T->g_last_w.end() ? -1 : it->second;
      }
      return T->last_w[key >> 20][key & 0xFFFFF];
    };
    for (long long k : R) p.push_back(lw(k));
    for (long long k : Wr) {
      p.push_back(lw(k));
      if (!(k >> 40)) {
        const auto& rd = T->readers[k >> 20][k & 0xFFFFF];
        p.insert(p.end(), rd.begin(), rd.end());
      }
    }
    std::sort(p.begin(), p.end());
    p.erase(std::unique(p.begin(), p.end()), p.end());
    if (!p.empty() && p.front() < 0) p.erase(p.begin());
    return p;
  }

  void record(int t, const std::vector<long long>& R, const std::vector<long long>& Wr) {
    for (long long k : Wr) {
      if (k >> 40) {
        T->g_last_w[k] = t;
      } else {
        T->last_w[k >> 20][k & 0xFFFFF] = t;
        T->readers[k >> 20][k & 0xFFFFF].clear();
      }
    }
    for (long long k : R)
      if (!(k >> 40)) {
        auto& rd = T->readers[k >> 20][k & 0xFFFFF];
        if (rd.empty() || rd.back() != t) rd.push_back(t);
      }
  }

  // Appends an op with the given predecessors (op numbers within the item);
  // its values go to the item's value region now.
  void raw(OpHdr h, const std::vector<int>& preds, const std::vector<uint16_t>& idx,
           const std::vector<double>& vals) {
    const int t = next_op++;
    OpRec r;
    if (!vals.empty()) {
      const size_t vb = pad16(vs * vals.size());
      h.vref = (uint32_t)(values->size() / 16);  // relative to the item; rebased when items are joined
      const size_t at = values->size();
      values->resize(at + vb, 0);
      for (size_t i = 0; i < vals.size(); ++i) put_value(values->data() + at, prec, i, vals[i]);
    }
    r.h = h;
    r.idx = idx;
    r.preds = preds;
    for (int u : preds)
      if (u < 0 || u >= t) throw std::logic_error("predecessor out of range");
    if (plant_unmet && h.kind >= OP_SYN_INTERP && h.kind <= OP_ANA_INTERP) {
      r.planted = true;
      plant_unmet = false;
    }
    // estimated cycles of one warp, fitted to the sweep's cycle counters on
    // GB300 at l = 1024 (two value caps per precision): a compute op costs a
    // fixed part (setup, value copy wait, reduction, completion) plus a part
    // per value; a control op a part per precision, a fold (two node values
    // per element, from global memory) about 2.4 times as much
    const double M = h.M, K = h.K;
    const double fixed = prec == 0 ? 1650.0 : prec == 2 ? 2100.0 : 1800.0;
    const double per_value = prec == 0 ? 15.2 : prec == 2 ? 4.6 : 1.25;
    const double ctl = (prec == 0 ? 2300.0 : prec == 2 ? 3800.0 : 1700.0) * (h.kind == OP_FOLD ? 2.4 : 1.0);
    r.cost = (h.kind >= OP_SYN_INTERP && h.kind <= OP_ANA_INTERP) ? fixed + per_value * M * K : ctl + 2.0 * M;
    r.stage = stage;
    ops.push_back(std::move(r));
  }

  // Opens a work item: the kernel's item barrier orders it after everything
  // before, so the tracker starts empty.
  void open_item(int npos) {
    positions = npos;
    next_op = 0;
    cursor = 0;
    base = 0;
    ops.clear();
    T->reset(positions);
  }

  void write(OpHdr h, const std::vector<uint16_t>& idx, const std::vector<double>& vals) {
    if (wide && base) throw std::logic_error("a wide stream places its one block at 0");
    // shift the op's vector positions to the block's base (control ops whose
    // offsets also index coefficients or node rows carry it in a0)
    switch (h.kind) {
      case OP_GATHER:
      case OP_SCATTER:
      case OP_FOLD:
        h.a0 = (uint16_t)(h.a0 | (base << 1));
        break;
      case OP_CLEAR:
        h.oo = (uint16_t)(h.oo + base);
        break;
      case OP_SYN_INTERP:
      case OP_DENSE:
      case OP_ANA_INTERP:
        h.io = (uint16_t)(h.io + base);
        h.oo = (uint16_t)(h.oo + base);
        break;
      case OP_DENSE_G:
        h.io = (uint16_t)(h.io + base);
        break;
      default:
        break;
    }
    std::vector<long long> R, Wr;
    access(h, idx, R, Wr);
    std::vector<int> preds = preds_of(R, Wr);
    const int t = next_op;
    raw(h, preds, idx, vals);
    record(t, R, Wr);
  }

  // A control op over [start, start + count), split into up to kCtlPieces warp tasks.
  void control(OpHdr base, int start, int count) {
    if (count <= 0) return;
    const int pieces = std::max(1, std::min(kCtlPieces, (count + 63) / 64));
    for (int q = 0; q < pieces; ++q) {
      const int a = start + (int)((long long)count * q / pieces);
      const int b = start + (int)((long long)count * (q + 1) / pieces);
      if (b <= a) continue;
      OpHdr h = base;
      h.M = (uint16_t)(b - a);
      set_io_oo(h, a, a);
      write(h, {}, {});
    }
  }

  // Size of the next piece of an op with `remaining` outputs whose record
  // and values for M outputs are allowed by ok(M).  A warp runs one piece
  // with one lane per output, or several lanes per output when the piece has
  // <= 16 outputs, so pieces of 32, 16, 8, ... outputs keep every lane busy;
  // the last piece takes the remainder.
  template <class F>
  int piece(int remaining, F ok) {
    if (remaining <= kMaxM && ok(remaining)) return remaining;
    for (int p2 = kMaxM; p2 >= 1; p2 /= 2)
      if (p2 <= remaining && ok(p2)) return p2;
    throw std::logic_error("op does not fit a record chunk and a staging slot");
  }

  // The piece sizes of an op with n outputs over K inputs, the first piece
  // allowed by ok_first(M), the others by ok(M).  Float64 and float32 take
  // the pieces of piece().  The split format's ops cost mostly a fixed part
  // (its reduction trees and per-op latency), so it takes the partition that
  // minimises an estimate of the warp's cycles per piece: 1800 fixed, 147
  // per inner step (ceil(K / ks) steps with ks = floor(32 / M) lanes per
  // output) and 280 per level of the reduction tree, the per-step figure
  // being the fitted cost per value of a full warp (4.6 x 32).
  template <class F1, class F2>
  std::vector<int> pieces(int n, int K, F1 ok_first, F2 ok) {
    std::vector<int> out;
    if (n <= 0) return out;
    if (prec != 2) {
      for (int o0 = 0; o0 < n;) {
        const int mp = o0 == 0 ? piece(n, ok_first) : piece(n - o0, ok);
        out.push_back(mp);
        o0 += mp;
      }
      return out;
    }
    auto t = [&](int M) {
      const int ks = kMaxM / M;
      int levels = 0;
      while ((1 << levels) < ks) ++levels;
      return 1800.0 + 147.0 * ((K + ks - 1) / ks) + 280.0 * levels;
    };
    // best[j]: the cheapest cover of the last j outputs by pieces allowed by ok
    const double inf = 1e300;
    std::vector<double> best(n + 1, inf);
    std::vector<int> pick(n + 1, 0);
    best[0] = 0.0;
    for (int j = 1; j <= n; ++j)
      for (int M = 1; M <= std::min(kMaxM, j); ++M)
        if (best[j - M] < inf && ok(M) && best[j - M] + t(M) < best[j]) {
          best[j] = best[j - M] + t(M);
          pick[j] = M;
        }
    int first = 0;
    double bf = inf;
    for (int M = 1; M <= std::min(kMaxM, n); ++M)
      if (best[n - M] < inf && ok_first(M) && t(M) + best[n - M] < bf) {
        bf = t(M) + best[n - M];
        first = M;
      }
    if (first == 0) throw std::logic_error("op does not fit a record chunk and a staging slot");
    out.push_back(first);
    for (int j = n - first; j > 0; j -= pick[j]) out.push_back(pick[j]);
    return out;
  }

  // y[oo + o] = z[io + skel[o]] + sum_s T[s][o] z[io + red[s]]
  void syn_interp(const IdBlock& b, uint8_t in_buf, uint8_t out_buf) {
    const int k = b.k, K = b.nin - b.k;
    auto ok = [&](int M) { return fits((size_t)K + M, (size_t)K * M); };
    int o0 = 0;
    for (const int mp : pieces(k, K, ok, ok)) {
      OpHdr h = hdr(OP_SYN_INTERP);
      h.in_buf = in_buf;
      h.out_buf = out_buf;
      h.M = (uint16_t)mp;
      h.K = (uint16_t)K;
      h.nskel = (uint16_t)mp;
      set_io_oo(h, b.in_off, b.out_off + o0);
      std::vector<uint16_t> idx(b.red.begin(), b.red.end());
      idx.insert(idx.end(), b.skel.begin() + o0, b.skel.begin() + o0 + mp);
      std::vector<double> vals((size_t)K * mp);
      for (int s = 0; s < K; ++s)
        for (int o = 0; o < mp; ++o) vals[(size_t)s * mp + o] = b.T[(size_t)s * k + o0 + o];
      write(h, idx, vals);
      o0 += mp;
    }
  }

  // out[oo + o] = sum_s V(s, o) in[io + s] (kind DENSE or DENSE_G)
  template <class GetV>
  void dense(uint8_t kind, uint8_t flags, int M, int K, GetV getv, uint8_t in_buf, int io, uint8_t out_buf, int oo,
             int m = 0) {
    auto ok = [&](int Mp) { return fits(0, (size_t)K * Mp); };
    int o0 = 0;
    for (const int mp : pieces(M, K, ok, ok)) {
      OpHdr h = hdr(kind, flags);
      h.in_buf = in_buf;
      h.out_buf = out_buf;
      h.M = (uint16_t)mp;
      h.K = (uint16_t)K;
      set_io_oo(h, io, oo + o0);
      if (!wide) h.a1 = (uint32_t)m;
      std::vector<double> vals((size_t)K * mp);
      for (int s = 0; s < K; ++s)
        for (int o = 0; o < mp; ++o) vals[(size_t)s * mp + o] = getv(s, o0 + o);
      write(h, {}, vals);
      o0 += mp;
    }
  }

  // z[oo + red[o]] (= or +=) sum_t T[o][t] y[io + t]; z[oo + skel[t]] (= or +=) y[io + t]
  void ana_interp(const IdBlock& b, uint8_t in_buf, uint8_t out_buf, bool accum) {
    const int k = b.k, nred = b.nin - b.k;
    if (k == 0) return;
    // the first op also carries the skeleton pass-through (k more indices);
    // with no redundant rows it is that alone
    std::vector<int> ps = pieces(
        nred, k, [&](int M) { return fits((size_t)M + k, (size_t)k * M); },
        [&](int M) { return fits((size_t)M, (size_t)k * M); });
    if (ps.empty()) {
      if (!fits((size_t)k, 0)) throw std::logic_error("skeleton pass-through does not fit a record chunk");
      ps.push_back(0);
    }
    bool skel_done = false;
    int o0 = 0;
    for (const int mp : ps) {
      OpHdr h = hdr(OP_ANA_INTERP, (uint8_t)((skel_done ? 0 : F_SKEL) | (accum ? F_ACCUM : 0)));
      h.in_buf = in_buf;
      h.out_buf = out_buf;
      h.M = (uint16_t)mp;
      h.K = (uint16_t)k;
      h.nskel = (uint16_t)(skel_done ? 0 : k);
      set_io_oo(h, b.out_off, b.in_off);
      std::vector<uint16_t> idx(b.red.begin() + o0, b.red.begin() + o0 + mp);
      if (!skel_done) idx.insert(idx.end(), b.skel.begin(), b.skel.end());
      std::vector<double> vals((size_t)k * mp);
      for (int t = 0; t < k; ++t)
        for (int o = 0; o < mp; ++o) vals[(size_t)t * mp + o] = b.T[(size_t)(o0 + o) * k + t];
      write(h, idx, vals);
      skel_done = true;
      o0 += mp;
    }
  }
};

// Shared vectors: both parities of an order use the pair (A, B) = (0, 1), one
// parity after the other, levels alternating between them.
constexpr uint8_t kBufA = 0, kBufB = 1;
inline uint8_t level_buf(int j) { return (j & 1) ? kBufB : kBufA; }
inline uint8_t other_buf(uint8_t b) { return (uint8_t)(b ^ 1); }

std::vector<const IdBlock*> blocks_at(const UnitFact& U, int j) {
  std::vector<const IdBlock*> v;
  for (const auto& b : U.blocks)
    if (b.level == j) v.push_back(&b);
  // largest first: the warps of a CTA then finish a level together
  std::stable_sort(v.begin(), v.end(), [](const IdBlock* a, const IdBlock* b) {
    return (long long)a->k * (a->nin - a->k + 1) > (long long)b->k * (b->nin - b->k + 1);
  });
  return v;
}

using Stage = std::function<void(Emitter&)>;

// Vector positions a parity block uses in either direction: its columns, its
// kept rows and every butterfly level.
int unit_width(const UnitFact& U) {
  int w = std::max(U.n, U.rows);
  for (int x : U.width) w = std::max(w, x);
  return w;
}

// Appends the ops of order m to the emitter's current work item.
//
// The blocks factor A_ij = sqrt(2 w_i) P-bar(x_i) over the positive nodes:
// the synthesis divides the rows by sqrt(2 w_i) (E_i and O_i at x_i), the
// analysis multiplies them by sqrt(w_i / 2) (the weighted, folded sums).  A
// single-block (gj) plan applies its block A = diag(sqrt(rho)) P-bar as it
// is (eqs. transform and transform2: forward A, inverse A^T), so both
// scales are 1; its one parity neither accumulates nor unfolds.
void emit_unit(PlanHost& P, int prec, int dir, int m, Emitter& E) {
  const int l = P.l;
  const std::vector<UnitFact>& F = (prec == 1) ? P.fact32 : P.fact64;
  std::vector<double> inv_sq2w(l, 1.0), sqw2(l, 1.0);
  if (!P.gj)
    for (int i = 0; i < l; ++i) {
      inv_sq2w[i] = 1.0 / std::sqrt(2.0 * P.w[l + i]);
      sqw2[i] = std::sqrt(0.5 * P.w[l + i]);
    }
  // the first parity with columns writes the node rows, the other adds
  const int first_p = F[(size_t)m * 2].n > 0 ? 0 : 1;
  std::vector<Stage> st[2];
  if (dir == 0) {
    // synthesis: gather, butterfly levels, then the final blocks write node
    // values: the even parity first (G = E), the odd parity after it (G +-= O)
    Stage fin[2];
    for (int p = 0; p < 2; ++p) {
      const UnitFact& U = F[(size_t)m * 2 + p];
      if (U.n == 0) continue;
      const uint8_t A = kBufA;
      const uint8_t gflags = p != first_p ? F_ACCUM : 0;
      st[p].push_back([&U, A, p, m](Emitter& E) {
        OpHdr g = E.hdr(OP_GATHER);
        g.a0 = (uint16_t)p;
        g.a1 = (uint32_t)m;
        g.out_buf = A;
        E.control(g, 0, U.n);
      });
      if (U.rows > 0 && !U.direct) {
        for (int j = 1; j <= U.levels + 1; ++j)
          st[p].push_back([&U, j, p](Emitter& E) {
            for (const IdBlock* b : blocks_at(U, j))
              if (b->k > 0) E.syn_interp(*b, j == 1 ? kBufA : level_buf(j - 1), level_buf(j));
          });
      }
      fin[p] = [&U, A, p, m, l, gflags, first_p, &inv_sq2w](Emitter& E) {
        if (U.rows > 0 && U.direct) {
          // E_i = sum_j P-bar(x_i) x_j: weighted values divided by sqrt(2 w_i)
          E.dense(OP_DENSE_G, gflags, U.rows, U.n,
                  [&](int s, int o) { return U.D[(size_t)s * U.rows + o] * inv_sq2w[o]; }, A, 0, A, 0, m);
        } else if (U.rows > 0) {
          const uint8_t top = level_buf(U.levels + 1);
          std::vector<const FinalBlock*> fs;
          for (const auto& f : U.finals) fs.push_back(&f);
          std::stable_sort(fs.begin(), fs.end(), [](const FinalBlock* a, const FinalBlock* b) {
            return (long long)a->k * (a->r1 - a->r0) > (long long)b->k * (b->r1 - b->r0);
          });
          for (const FinalBlock* f : fs) {
            const int h = f->r1 - f->r0;
            if (f->k == 0 && p == 1) continue;  // adds nothing
            E.dense(OP_DENSE_G, gflags, h, f->k,
                    [&](int s, int o) { return f->S[(size_t)s * h + o] * inv_sq2w[f->r0 + o]; }, top, f->in_off,
                    A, f->r0, m);
          }
        }
        if (p == first_p && U.rows < l) {
          // node rows past the kept ones hold no even part
          OpHdr z = E.hdr(OP_GZERO);
          z.a1 = (uint32_t)m;
          E.control(z, U.rows, l - U.rows);
        }
      };
    }
    // each parity block at its own place in the shared vectors: where both
    // fit, the parities run concurrently; otherwise the tracker orders the
    // next block's writes after this one's final reads
    for (int p = 0; p < 2; ++p) {
      E.place(unit_width(F[(size_t)m * 2 + p]));
      for (const Stage& sg : st[p]) {
        ++E.stage;
        sg(E);
      }
      if (fin[p]) {
        ++E.stage;
        fin[p](E);
      }
    }
  } else {
    for (int p = 0; p < 2; ++p) {
      const UnitFact& U = F[(size_t)m * 2 + p];
      if (U.n == 0) continue;
      const uint8_t A = kBufA, B = kBufB;
      if (U.rows == 0) {
        st[p].push_back([&U, A](Emitter& E) {
          OpHdr c = E.hdr(OP_CLEAR);
          c.out_buf = A;
          E.control(c, 0, U.n);
        });
      } else {
        const uint8_t top = U.direct ? A : level_buf(U.levels + 1);
        const uint8_t ubuf = U.direct ? B : other_buf(top);
        st[p].push_back([&U, ubuf, p, m](Emitter& E) {
          OpHdr f = E.hdr(OP_FOLD);
          f.a0 = (uint16_t)p;
          f.a1 = (uint32_t)m;
          f.out_buf = ubuf;
          E.control(f, 0, U.rows);
        });
        if (U.direct) {
          // x_j = sum_i w_i P-bar(x_i) u_i: weighted values times sqrt(w_i / 2)
          st[p].push_back([&U, ubuf, A, &sqw2](Emitter& E) {
            E.dense(OP_DENSE, 0, U.n, U.rows, [&](int s, int o) { return U.D[(size_t)o * U.rows + s] * sqw2[s]; },
                    ubuf, 0, A, 0);
          });
        } else {
          st[p].push_back([&U, ubuf, top, &sqw2](Emitter& E) {
            for (const auto& fb : U.finals) {
              if (fb.k == 0) continue;
              const int h = fb.r1 - fb.r0;
              E.dense(OP_DENSE, 0, fb.k, h, [&](int s, int o) { return fb.S[(size_t)o * h + s] * sqw2[fb.r0 + s]; },
                      ubuf, fb.r0, top, fb.in_off);
            }
          });
          for (int j = U.levels + 1; j >= 2; --j) {
            // blocks of level j come in pairs (top band 2b, bottom band 2b+1) sharing one input
            // vector z of level j-1: the top halves overwrite z, then the bottom halves add
            const uint8_t src = level_buf(j), dst = level_buf(j - 1);
            auto tops = std::make_shared<std::vector<const IdBlock*>>();
            auto second = std::make_shared<std::vector<const IdBlock*>>();
            std::vector<const IdBlock*> bots;
            for (const IdBlock* b : blocks_at(U, j)) (b->band % 2 == 0 ? *tops : bots).push_back(b);
            auto firsts = std::make_shared<std::vector<std::pair<const IdBlock*, int>>>();  // (block or top, mode)
            for (const IdBlock* t : *tops) {
              const IdBlock* bp = nullptr;
              for (const IdBlock* b : bots)
                if (b->band == t->band + 1 && b->group == t->group) bp = b;
              if (t->k > 0) {
                firsts->push_back({t, 0});
                if (bp && bp->k > 0) second->push_back(bp);
              } else if (bp && bp->k > 0) {
                firsts->push_back({bp, 0});
              } else if (t->nin > 0) {
                firsts->push_back({t, 1});  // nothing interpolates into z: clear it
              }
            }
            st[p].push_back([firsts, src, dst](Emitter& E) {
              for (const auto& pr : *firsts) {
                if (pr.second == 0) {
                  E.ana_interp(*pr.first, src, dst, false);
                } else {
                  OpHdr c = E.hdr(OP_CLEAR);
                  c.out_buf = dst;
                  E.control(c, pr.first->in_off, pr.first->nin);
                }
              }
            });
            if (!second->empty())
              st[p].push_back([second, src, dst](Emitter& E) {
                for (const IdBlock* b : *second) E.ana_interp(*b, src, dst, true);
              });
          }
          st[p].push_back([&U, A, B](Emitter& E) {
            for (const IdBlock* b : blocks_at(U, 1)) {
              if (b->k > 0) {
                E.ana_interp(*b, B, A, false);
              } else {
                OpHdr c = E.hdr(OP_CLEAR);
                c.out_buf = A;
                E.control(c, b->in_off, b->nin);
              }
            }
          });
        }
      }
      st[p].push_back([&U, A, p, m](Emitter& E) {
        OpHdr s = E.hdr(OP_SCATTER);
        s.a0 = (uint16_t)p;
        s.a1 = (uint32_t)m;
        s.in_buf = A;
        E.control(s, 0, U.n);
      });
    }
    for (int p = 0; p < 2; ++p) {
      E.place(unit_width(F[(size_t)m * 2 + p]));
      for (const Stage& sg : st[p]) {
        ++E.stage;
        sg(E);
      }
    }
  }
}

// Schedules the ops of one work item onto nw warps and encodes the item
// (ItemHeader, WarpRange[nw], then each warp's record stream in chunks of
// `chunk` bytes; see sht_stream.h).  Event-driven list scheduling on the
// estimated costs: whenever a warp falls free, it takes, among the ops whose
// predecessors are all scheduled, the most critical one that can start now
// (the longest estimated path to the end of the item), or else the one that
// can start soonest.  An op is scheduled only after its predecessors, so each
// warp's list is a topological order and a wait on another warp's earlier
// position can never close a cycle.  Returns the item bytes (a multiple of 16).
void encode_item(const std::vector<OpRec>& ops, int nw, size_t chunk, std::vector<uint8_t>& out) {
  const int n = (int)ops.size();
  std::vector<int> warp(n), pos(n), cnt(nw, 0), order;
  order.reserve(n);
  {
    // successors and bottom levels (longest estimated path to the item's end)
    std::vector<std::vector<int>> succ(n);
    std::vector<int> npend(n, 0);
    for (int t = 0; t < n; ++t) {
      npend[t] = (int)ops[t].preds.size();
      for (int u : ops[t].preds) succ[u].push_back(t);
    }
    std::vector<double> blevel(n, 0.0);
    for (int t = n - 1; t >= 0; --t) {
      double b = 0;
      for (int v : succ[t]) b = std::max(b, blevel[v]);
      blevel[t] = ops[t].cost + b;
    }
    std::vector<double> ready_at(n, 0.0), wfree(nw, 0.0);
    std::vector<int> cand;
    for (int t = 0; t < n; ++t)
      if (npend[t] == 0) cand.push_back(t);
    for (int done = 0; done < n; ++done) {
      int w = 0;
      for (int v = 1; v < nw; ++v)
        if (wfree[v] < wfree[w]) w = v;
      const double now = wfree[w];
      // the most critical op that is ready now, else the one ready soonest
      int best = -1;
      bool best_ready = false;
      for (int i = 0; i < (int)cand.size(); ++i) {
        const int t = cand[i];
        const bool r = ready_at[t] <= now;
        if (best < 0) {
          best = i;
          best_ready = r;
          continue;
        }
        const int b = cand[best];
        bool better;
        if (r != best_ready) {
          better = r;
        } else if (r) {
          better = blevel[t] > blevel[b] || (blevel[t] == blevel[b] && t < b);
        } else {
          better = ready_at[t] < ready_at[b] || (ready_at[t] == ready_at[b] && blevel[t] > blevel[b]);
        }
        if (better) {
          best = i;
          best_ready = r;
        }
      }
      const int t = cand[best];
      cand[best] = cand.back();
      cand.pop_back();
      const double fin = std::max(now, ready_at[t]) + ops[t].cost;
      wfree[w] = fin;
      warp[t] = w;
      pos[t] = cnt[w]++;
      order.push_back(t);
      for (int v : succ[t]) {
        ready_at[v] = std::max(ready_at[v], fin);
        if (--npend[v] == 0) cand.push_back(v);
      }
    }
  }
  for (int w = 0; w < nw; ++w)
    if (cnt[w] > kMaxWarpOps) throw std::logic_error("work item has too many ops for one warp");
  // ops another warp waits for: their warps publish progress after them
  std::vector<char> waited_for(n, 0);
  {
    std::vector<int> last(nw);
    for (int t = 0; t < n; ++t) {
      std::fill(last.begin(), last.end(), -1);
      for (int u : ops[t].preds)
        if (warp[u] != warp[t] && (last[warp[u]] < 0 || pos[u] > pos[last[warp[u]]])) last[warp[u]] = u;
      for (int v = 0; v < nw; ++v)
        if (last[v] >= 0) waited_for[last[v]] = 1;
    }
  }
  std::vector<std::vector<uint8_t>> st(nw);
  std::vector<int> need(nw);
  for (int t : order) {
    const int w = warp[t];
    std::fill(need.begin(), need.end(), -1);
    for (int u : ops[t].preds)
      if (warp[u] != w) need[warp[u]] = std::max(need[warp[u]], pos[u]);
    std::vector<uint16_t> all;
    for (int v = 0; v < nw; ++v)
      if (need[v] >= 0) all.push_back((uint16_t)((v << kPredPosBits) | need[v]));
    if (ops[t].planted) all.push_back((uint16_t)((w << kPredPosBits) | pos[t]));  // itself: never complete
    OpHdr h = ops[t].h;
    if (waited_for[t]) h.flags |= F_PUBLISH;
    h.npred = (uint16_t)all.size();
    all.insert(all.end(), ops[t].idx.begin(), ops[t].idx.end());
    const size_t ib = pad16(2 * all.size());
    h.idx16 = (uint16_t)(ib / 16);
    h.bytes = (uint32_t)(sizeof(OpHdr) + ib);
    if (h.bytes > chunk) throw std::logic_error("record larger than a chunk");
    std::vector<uint8_t>& B = st[w];
    const size_t in_chunk = B.size() % chunk;
    if (in_chunk && in_chunk + h.bytes > chunk) B.resize(B.size() + (chunk - in_chunk), 0);  // zero header: chunk ends
    const size_t at = B.size();
    B.resize(at + h.bytes, 0);
    std::memcpy(B.data() + at, &h, sizeof(OpHdr));
    if (!all.empty()) std::memcpy(B.data() + at + sizeof(OpHdr), all.data(), 2 * all.size());
  }
  const size_t head = pad16(sizeof(ItemHeader) + sizeof(WarpRange) * (size_t)nw);
  size_t total = head;
  for (int w = 0; w < nw; ++w) total += st[w].size();
  out.assign(total, 0);
  ItemHeader ih{};
  ih.magic = kItemMagic;
  ih.nw = (uint16_t)nw;
  ih.n_ops = (uint32_t)n;
  std::memcpy(out.data(), &ih, sizeof(ih));
  size_t off = head;
  for (int w = 0; w < nw; ++w) {
    WarpRange r{(uint32_t)off, (uint32_t)st[w].size()};
    std::memcpy(out.data() + sizeof(ItemHeader) + sizeof(WarpRange) * (size_t)w, &r, sizeof(r));
    if (!st[w].empty()) std::memcpy(out.data() + off, st[w].data(), st[w].size());
    off += st[w].size();
  }
}

// Calls fn(header) for every record of an encoded item.
template <class Fn>
void for_each_record(uint8_t* item, size_t chunk, Fn fn) {
  ItemHeader ih;
  std::memcpy(&ih, item, sizeof(ih));
  for (int w = 0; w < ih.nw; ++w) {
    WarpRange r;
    std::memcpy(&r, item + sizeof(ItemHeader) + sizeof(WarpRange) * (size_t)w, sizeof(r));
    size_t p = 0;
    while (p < r.bytes) {
      OpHdr* h = reinterpret_cast<OpHdr*>(item + r.off + p);
      if (h->bytes == 0) {
        p = (p / chunk + 1) * chunk;
        continue;
      }
      fn(h);
      p += h->bytes;
    }
  }
}

}  // namespace

namespace {

// Level-by-level streams of a single-block (gj) plan.  The block is emitted
// as one order (emit_unit), then its ops are cut at the stage boundaries:
// the ops of one stage (the gather, one butterfly level, the final blocks,
// ...) touch disjoint vector elements, so every stage becomes one launch of
// independent work items, its vectors in global memory and its items spread
// over the GPU; the launches run in stage order.  An op whose predecessor
// lies in its own stage would break that, and is refused.
void emit_gj_streams(PlanHost& P, int prec) {
  const std::vector<UnitFact>& F = (prec == 1) ? P.fact32 : P.fact64;
  if (F.size() != 2) throw std::logic_error("single-block plan without its factorization");
  const size_t CH = (size_t)P.page_bytes;
  const int NW = P.sched_warps;
  const UnitFact& U = F[(size_t)P.gj_p];
  const int positions = unit_width(U) + 1;
  if (positions > (1 << 20)) throw std::runtime_error("block too wide: vector positions exceed 20 bits");
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<uint8_t> vals;
    Emitter E(prec);
    Tracker T;
    E.T = &T;
    E.l = P.l;
    E.values = &vals;
    E.slot_values = P.slot_values_for(prec);
    E.chunk = CH;
    E.pool = positions - 1;
    E.wide = true;
    E.open_item(positions);
    emit_unit(P, prec, dir, 0, E);
    const std::vector<OpRec>& ops = E.ops;
    for (const OpRec& r : ops)
      for (int u : r.preds)
        if (ops[(size_t)u].stage >= r.stage) throw std::logic_error("dependency inside a stage");
    Stream& S = P.streams[prec][dir];
    S.units.clear();
    S.stage_begin.clear();
    std::vector<uint8_t> bytes, item;
    constexpr double kGuideCtas = 2 * 152;  // items per stage to aim for (two per SM of a GB300)
    constexpr double kMinItemCost = 40000;  // estimated warp cycles below which an item is not split
    const size_t max_ops = (size_t)NW * 256;
    size_t t = 0;
    while (t < ops.size()) {
      size_t t1 = t;
      double cost = 0;
      while (t1 < ops.size() && ops[t1].stage == ops[t].stage) cost += ops[t1++].cost;
      const double target = std::max(cost / kGuideCtas, kMinItemCost);
      S.stage_begin.push_back((uint32_t)S.units.size());
      std::vector<OpRec> cur;
      double cc = 0;
      auto flush = [&]() {
        encode_item(cur, NW, CH, item);
        UnitEntry e;
        e.off16 = bytes.size() / 16;
        e.len16 = (uint32_t)(item.size() / 16);
        e.m = (uint32_t)P.gj_m;
        S.units.push_back(e);
        bytes.insert(bytes.end(), item.begin(), item.end());
        cur.clear();
        cc = 0;
      };
      for (size_t u = t; u < t1; ++u) {
        if (!cur.empty() && (cc + ops[u].cost > target || cur.size() >= max_ops)) flush();
        cur.push_back(ops[u]);
        cur.back().preds.clear();  // earlier stages: ordered by the launches
        cc += ops[u].cost;
      }
      if (!cur.empty()) flush();
      t = t1;
    }
    S.stage_begin.push_back((uint32_t)S.units.size());
    if (vals.size() / 16 > 0xFFFFFFFFull) throw std::runtime_error("value region exceeds 64 GB");
    ByteBuf().swap(S.bytes);
    ByteBuf().swap(S.values);
    S.bytes.resize(std::max<size_t>(bytes.size(), 16), 0);
    if (!bytes.empty()) std::memcpy(S.bytes.data(), bytes.data(), bytes.size());
    S.values.resize(vals.size());
    if (!vals.empty()) std::memcpy(S.values.data(), vals.data(), vals.size());
    S.max_buf_ab = positions - 1;
    S.num_vecs = 2;
  }
  P.built[prec] = true;
}

}  // namespace

void build_gj_factorization(PlanHost& P, bool fp32) {
  std::vector<UnitFact>& out = fp32 ? P.fact32 : P.fact64;
  out.assign(2, UnitFact());
  out[(size_t)P.gj_p] = factor_single_unit(P, P.gj_m, P.gj_p, fp32 ? P.eps_fp32 : P.eps_id);
}

void emit_streams(PlanHost& P, int prec) {
  if (P.gj) {
    emit_gj_streams(P, prec);
    return;
  }
  const int L = 2 * P.l;
  const std::vector<UnitFact>& F = (prec == 1) ? P.fact32 : P.fact64;
  const size_t CH = (size_t)P.page_bytes;
  const int NW = P.sched_warps;
  int positions = 1;
  for (const UnitFact& U : F) {
    positions = std::max({positions, U.n, U.rows});
    for (int wdt : U.width) positions = std::max(positions, wdt);
  }
  positions += 1;
  for (int dir = 0; dir < 2; ++dir) {
    int nt = P.num_threads > 0 ? P.num_threads : (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt, 256));
    auto run_parallel = [&](int count, auto&& body) {
      std::atomic<int> next(0);
      std::vector<std::string> errors(nt);
      auto worker = [&](int tid) {
        try {
          for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            body(i);
          }
        } catch (const std::exception& e) {
          errors[tid] = e.what();
          next.store(count);
        }
      };
      std::vector<std::thread> th;
      for (int t = 1; t < nt; ++t) th.emplace_back(worker, t);
      worker(0);
      for (auto& t : th) t.join();
      for (auto& e : errors)
        if (!e.empty()) throw std::runtime_error(e);
    };
    // emits a list of orders as one scheduled work item; returns its op count
    auto emit_item = [&](const std::vector<int>& ms, std::vector<uint8_t>& out, std::vector<uint8_t>& vals) -> int {
      Emitter E(prec);
      Tracker T;
      E.T = &T;
      E.l = P.l;
      E.values = &vals;
      E.plant_unmet = P.debug_unmet_dep && std::find(ms.begin(), ms.end(), 0) != ms.end();
      E.slot_values = P.slot_values_for(prec);
      E.chunk = CH;
      E.pool = positions - 1;
      E.open_item(positions);
      for (int m : ms) emit_unit(P, prec, dir, m, E);
      encode_item(E.ops, NW, CH, out);
      return E.next_op;
    };
    // pass 1: every order alone (its size decides the packing)
    std::vector<std::vector<uint8_t>> per(L), per_vals(L);
    std::vector<int> nops(L);
    run_parallel(L, [&](int m) { nops[m] = emit_item({m}, per[m], per_vals[m]); });
    // work of an order: its record and value bytes, in units of 1 KB
    auto work_kb = [&](int m) { return (per[m].size() + per_vals[m].size() + 1023) / 1024; };
    size_t total_kb = 0;
    for (int m = 0; m < L; ++m) total_kb += work_kb(m);
    // Work items: orders in decreasing size, packed with guided sizes: an
    // item takes about remaining / (2 x 152) of the work not yet packed
    // (152: the SMs of the GB300 the persistent kernel runs one CTA on each),
    // at least 32 KB, so the queue starts with large items and ends with
    // small ones that even out the CTAs' finishing times; more than one order
    // per item where they fit, so the tail of one overlaps the next; at most
    // kMaxWarpOps ops (so no warp's position overflows a pred entry).
    constexpr size_t kGuideCtas = 2 * 152;
    std::vector<int> order(L);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work_kb(a) > work_kb(b); });
    std::vector<std::vector<int>> items;
    std::vector<int> cur;
    size_t cur_kb = 0, remaining = total_kb;
    int cur_ops = 0;
    size_t target = std::max<size_t>(32, remaining / kGuideCtas);
    for (int m : order) {
      const size_t kb = work_kb(m);
      if (!cur.empty() && (cur_kb + kb > target || cur_ops + nops[m] > kMaxWarpOps)) {
        items.push_back(cur);
        remaining -= std::min(remaining, cur_kb);
        target = std::max<size_t>(32, remaining / kGuideCtas);
        cur.clear();
        cur_kb = 0;
        cur_ops = 0;
      }
      cur.push_back(m);
      cur_kb += kb;
      cur_ops += nops[m];
    }
    if (!cur.empty()) items.push_back(cur);
    std::vector<std::vector<uint8_t>> item_bytes(items.size()), item_vals(items.size());
    run_parallel((int)items.size(), [&](int it) {
      if (items[it].size() == 1) {
        item_bytes[it].swap(per[items[it][0]]);
        item_vals[it].swap(per_vals[items[it][0]]);
        return;
      }
      emit_item(items[it], item_bytes[it], item_vals[it]);
    });
    std::vector<int> iorder(items.size());
    std::iota(iorder.begin(), iorder.end(), 0);
    std::stable_sort(iorder.begin(), iorder.end(), [&](int a, int b) {
      return item_bytes[a].size() + item_vals[a].size() > item_bytes[b].size() + item_vals[b].size();
    });

    Stream& S = P.streams[prec][dir];
    S.units.clear();
    // offsets of every item in the joined record and value regions
    std::vector<size_t> byte_off(items.size()), val_off(items.size());
    size_t nbytes = 0, nvals = 0;
    for (int it : iorder) {
      byte_off[it] = nbytes;
      val_off[it] = nvals;
      UnitEntry e;
      e.off16 = nbytes / 16;
      e.len16 = (uint32_t)(item_bytes[it].size() / 16);
      e.m = (uint32_t)items[it][0];
      S.units.push_back(e);
      nbytes += item_bytes[it].size();
      nvals += item_vals[it].size();
    }
    if (nvals / 16 > 0xFFFFFFFFull) throw std::runtime_error("value region exceeds 64 GB");
    ByteBuf().swap(S.bytes);
    ByteBuf().swap(S.values);
    S.bytes.resize(std::max<size_t>(nbytes, 16));
    S.values.resize(nvals);
    // rebase each item's value references onto the joined value region and
    // copy it into place, items in parallel
    run_parallel((int)items.size(), [&](int it) {
      const uint32_t base16 = (uint32_t)(val_off[it] / 16);
      std::vector<uint8_t>& B = item_bytes[it];
      if (base16 && !item_vals[it].empty())
        for_each_record(B.data(), CH, [&](OpHdr* h) {
          if (h->kind >= OP_SYN_INTERP && h->kind <= OP_ANA_INTERP) h->vref += base16;
        });
      if (!B.empty()) std::memcpy(S.bytes.data() + byte_off[it], B.data(), B.size());
      if (!item_vals[it].empty())
        std::memcpy(S.values.data() + val_off[it], item_vals[it].data(), item_vals[it].size());
      std::vector<uint8_t>().swap(B);
      std::vector<uint8_t>().swap(item_vals[it]);
    });
    // blocks are placed anywhere in the first positions - 1 elements
    S.max_buf_ab = positions - 1;
    S.num_vecs = 2;
  }
  P.built[prec] = true;
}

}  // namespace sht
