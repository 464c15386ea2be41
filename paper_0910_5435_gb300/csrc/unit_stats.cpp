// unit_stats.cpp -- rank statistics and accuracy of the butterfly of ONE
// parity block, at bandlimits beyond what a whole plan holds.
//
// For m = 0 and p = 0 the block A_{ij} = sqrt(2 w_{l+i}) P-bar^0_{2j}(x_{l+i})
// (i, j < l) is the matrix of the paper's even-degree transform with n = l
// (Section 4, eqs. transform / evens with the Gauss-Legendre nodes; its
// rho_i equal 2 w_{l+i}), so its ID ranks and errors can be set beside the
// paper's Table small_time / small_pre.  The paper's general-m matrices (eq.
// transform at the n positive zeros of P-bar^m_{m+2n} with the weights of
// Lemma quadratures, and eq. transform2 for odd degrees) are built here too,
// at nodes computed from the x^2 recurrence (gauss_jacobi_nodes), for its
// Tables evens and odds.  Host only, float64.
//
// The factorization is applied on the host exactly as the butterfly defines
// it (Section 2.2 eqs. 1-6: y = z[skel] + T z[red] level by level, then the
// stored skeleton columns of each row band, Section 3), and its transpose
// for the inverse (Section 2.2, remark after Figure multi).  The direct
// products stream the columns of A with the same x^2 recurrence, so no
// l x n array is stored.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <exception>
#include <new>
#include <thread>
#include <vector>

#include "../../include/sht.h"
#include "plan_host.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// SplitMix64 (Steele, Lea and Flood 2014): uniform doubles in (-1, 1).
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform_pm1() { return ((double)(next() >> 11) + 0.5) * (2.0 / 9007199254740992.0) - 1.0; }
};

std::vector<double> unit_vector(size_t n, uint64_t seed) {
  SplitMix64 g{seed};
  std::vector<double> v(n);
  double s = 0;
  for (double& x : v) {
    x = g.uniform_pm1();
    s += x * x;
  }
  const double inv = s > 0 ? 1.0 / std::sqrt(s) : 0.0;
  for (double& x : v) x *= inv;
  return v;
}

// Blocks of each level, in any order (each block reads and writes its own ranges).
std::vector<std::vector<const sht::IdBlock*>> by_level(const sht::UnitFact& U) {
  std::vector<std::vector<const sht::IdBlock*>> at(U.levels + 2);
  for (const auto& b : U.blocks) at[b.level].push_back(&b);
  return at;
}

// alpha = A beta through the factorization (alpha has l entries; trimmed rows 0).
std::vector<double> apply_forward(const sht::UnitFact& U, int l, const std::vector<double>& beta) {
  std::vector<double> alpha(l, 0.0);
  if (U.direct) {
    for (int j = 0; j < U.n; ++j)
      for (int i = 0; i < U.rows; ++i) alpha[i] += U.D[(size_t)j * U.rows + i] * beta[j];
    return alpha;
  }
  const int top = U.levels + 1;
  const auto at = by_level(U);
  std::vector<std::vector<double>> lay(top + 1);
  for (int j = 1; j <= top; ++j) {
    lay[j].assign(U.width[j], 0.0);
    for (const sht::IdBlock* b : at[j]) {
      const double* z = (j == 1) ? beta.data() + b->in_off : lay[j - 1].data() + b->in_off;
      const int k = b->k;
      for (int t = 0; t < k; ++t) {
        double y = z[b->skel[t]];
        for (size_t s = 0; s < b->red.size(); ++s) y += b->T[s * k + t] * z[b->red[s]];
        lay[j][b->out_off + t] = y;
      }
    }
  }
  for (const sht::FinalBlock& f : U.finals) {
    const int h = f.r1 - f.r0;
    for (int i = 0; i < h; ++i) {
      double a = 0;
      for (int t = 0; t < f.k; ++t) a += f.S[(size_t)t * h + i] * lay[top][f.in_off + t];
      alpha[f.r0 + i] = a;
    }
  }
  return alpha;
}

// nu = A^T mu through the transposed factorization.
std::vector<double> apply_transpose(const sht::UnitFact& U, const std::vector<double>& mu) {
  std::vector<double> nu(U.n, 0.0);
  if (U.direct) {
    for (int j = 0; j < U.n; ++j)
      for (int i = 0; i < U.rows; ++i) nu[j] += U.D[(size_t)j * U.rows + i] * mu[i];
    return nu;
  }
  const int top = U.levels + 1;
  const auto at = by_level(U);
  std::vector<std::vector<double>> lay(top + 1);
  for (int j = 1; j <= top; ++j) lay[j].assign(U.width[j], 0.0);
  for (const sht::FinalBlock& f : U.finals) {
    const int h = f.r1 - f.r0;
    for (int t = 0; t < f.k; ++t) {
      double y = 0;
      for (int i = 0; i < h; ++i) y += f.S[(size_t)t * h + i] * mu[f.r0 + i];
      lay[top][f.in_off + t] = y;
    }
  }
  for (int j = top; j >= 1; --j) {
    for (const sht::IdBlock* b : at[j]) {
      double* z = (j == 1) ? nu.data() + b->in_off : lay[j - 1].data() + b->in_off;
      const int k = b->k;
      for (int t = 0; t < k; ++t) {
        const double y = lay[j][b->out_off + t];
        z[b->skel[t]] += y;
        for (size_t s = 0; s < b->red.size(); ++s) z[b->red[s]] += b->T[s * k + t] * y;
      }
    }
  }
  return nu;
}

// Statistics of the butterfly of the block (m, parity) of P (nodes set).
sht_status unit_stats_of(sht::PlanHost& P, int m, int parity, double eps_id, double t_quad, unsigned long long seed,
                         sht_unit_stats* out) {
  const int l = P.l;
  const double t0 = now_s();
  const sht::UnitFact U = sht::factor_single_unit(P, m, parity, eps_id);
  const double t_comp = now_s() - t0;

  sht_unit_stats s{};
  s.l = l;
  s.m = m;
  s.parity = parity;
  s.n = U.n;
  s.rows_kept = U.rows;
  s.levels = U.levels;
  s.direct = U.direct ? 1 : 0;
  double sumk = 0, sumk2 = 0;
  for (const auto& b : U.blocks) {
    s.k_max = std::max(s.k_max, b.k);
    sumk += b.k;
    sumk2 += (double)b.k * b.k;
    for (double t : b.T) s.max_abs_T = std::max(s.max_abs_T, std::fabs(t));
  }
  s.n_blocks = (int)U.blocks.size();
  if (s.n_blocks) {
    s.k_avg = sumk / s.n_blocks;
    s.k_sigma = std::sqrt(std::max(0.0, sumk2 / s.n_blocks - s.k_avg * s.k_avg));
  }
  s.factor_values = U.values;
  s.dense_values = (long long)l * U.n;
  s.m_max_words = U.peak_words;
  s.t_quad = t_quad;
  s.t_comp = t_comp;

  // accuracy against the direct products, unit-norm U(-1, 1) inputs
  if (U.n > 0) {
    const std::vector<double> beta = unit_vector(U.n, seed);
    const std::vector<double> mu = unit_vector(l, seed + 1);
    std::vector<double> alpha_d(l, 0.0), nu_d(U.n, 0.0), col(l);
    sht::ColumnStream cs(P, m, parity, l);
    for (int j = 0; j < U.n; ++j) {
      cs.next(col.data());
      double dot = 0;
      for (int i = 0; i < l; ++i) {
        alpha_d[i] += col[i] * beta[j];
        dot += col[i] * mu[i];
      }
      nu_d[j] = dot;
    }
    const std::vector<double> alpha = apply_forward(U, l, beta);
    const std::vector<double> nu = apply_transpose(U, mu);
    for (int i = 0; i < l; ++i) s.eps_fwd = std::max(s.eps_fwd, std::fabs(alpha[i] - alpha_d[i]));
    for (int j = 0; j < U.n; ++j) s.eps_inv = std::max(s.eps_inv, std::fabs(nu[j] - nu_d[j]));
  }
  *out = s;
  return SHT_OK;
}

bool options_ok(const sht_plan_opts* opts, sht_plan_opts* o) {
  if (opts) {
    *o = *opts;
  } else {
    sht_plan_opts_default(o);
  }
  return o->leaf_cols >= 2 && o->leaf_cols <= 1024;
}

void apply_options(sht::PlanHost& P, const sht_plan_opts& o, double eps_id) {
  P.eps_id = eps_id;
  P.trim_eps = o.trim_eps < 0 ? eps_id : o.trim_eps;
  P.leaf_cols = o.leaf_cols;
  P.min_band_rows = o.min_band_rows > 0 ? o.min_band_rows : std::max(1, o.leaf_cols / 2);
}

}  // namespace

namespace sht {

// Nodes: the x^2 recurrence on the basis P-bar^m_{m+p+2j}, j < n, is the
// symmetric tridiagonal (Jacobi) matrix J with J_jj = d_{m+p+2j} and
// J_{j,j+1} = c_{m+p+2j} acting on t = x^2; the zeros in t of
// P-bar^m_{m+p+2n} are its eigenvalues.  Each eigenvalue is bracketed by
// Sturm-sequence bisection (Barth, Martin and Wilkinson 1967) and then
// refined by Newton's method on the three-term recurrence itself (which
// keeps full relative accuracy for the small t near x = 0).  Weights: the
// rows of sqrt(rho_i) P-bar^m_{m+p+2j}(x_i) are orthonormal (the matrix is
// orthogonal by Lemma quadratures), so rho_i = 1 / sum_{j<n} P-bar^m_{m+p+2j}(x_i)^2.
namespace {
// Runs body(i), i < count, on all hardware threads.
template <class F>
void parallel_for(int count, F&& body) {
  const int nt = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
  std::atomic<int> next(0);
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      body(i);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
}
}  // namespace

void gauss_jacobi_nodes(int m, int p, int n, std::vector<double>& x, std::vector<double>& sin_theta,
                        std::vector<double>& rho) {
  std::vector<double> a(n), b2(n, 0.0);
  for (int j = 0; j < n; ++j) {
    a[j] = rec_d(m + p + 2 * j, m);
    if (j + 1 < n) {
      const double c = rec_c(m + p + 2 * j, m);
      b2[j] = c * c;
    }
  }
  // number of eigenvalues below lam (negative pivots of J - lam I = L D L^T)
  auto below = [&](double lam) {
    int cnt = 0;
    double q = 1.0;
    for (int j = 0; j < n; ++j) {
      q = (a[j] - lam) - (j ? b2[j - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
    }
    return cnt;
  };
  std::vector<double> t(n), cc(n), cm(n);
  for (int j = 0; j < n; ++j) {
    const int kk = m + p + 2 * j;
    cc[j] = rec_c(kk, m);
    cm[j] = j ? rec_c(kk - 2, m) : 0.0;
  }
  // The eigenvalues are independent: chunks of consecutive indices run on
  // the host threads (within a chunk, each bracket starts at the previous
  // eigenvalue's lower end; a chunk starts at 0), so the results do not
  // depend on the number of threads.
  constexpr int kChunk = 64;
  const int nchunks = (n + kChunk - 1) / kChunk;
  parallel_for(nchunks, [&](int ch) {
    const int k0 = ch * kChunk, k1 = std::min(n, k0 + kChunk);
    double lo_prev = 0.0;
    for (int k = k0; k < k1; ++k) {
      double lo = lo_prev, hi = 1.0;
      for (int it = 0; it < 56 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) > k) hi = mid; else lo = mid;
      }
      lo_prev = lo;
      // Newton on the degree-n polynomial of the recurrence (value and
      // derivative, rescaled together against overflow)
      double tk = 0.5 * (lo + hi);
      for (int it = 0; it < 4; ++it) {
        double q0 = 0.0, dq0 = 0.0, q1 = 1.0, dq1 = 0.0;
        for (int j = 0; j < n; ++j) {
          const double q2 = ((tk - a[j]) * q1 - cm[j] * q0) / cc[j];
          const double dq2 = ((tk - a[j]) * dq1 + q1 - cm[j] * dq0) / cc[j];
          q0 = q1;
          dq0 = dq1;
          q1 = q2;
          dq1 = dq2;
          const double big = std::max(std::fabs(q1), std::fabs(dq1));
          if (big > 1e150) {
            q0 /= big;
            dq0 /= big;
            q1 /= big;
            dq1 /= big;
          }
        }
        if (dq1 == 0.0) break;
        const double step = q1 / dq1;
        tk -= step;
        if (std::fabs(step) <= 1e-17 * tk) break;
      }
      t[k] = tk;
    }
  });
  x.resize(n);
  sin_theta.resize(n);
  for (int k = 0; k < n; ++k) {
    x[k] = std::sqrt(t[k]);
    sin_theta[k] = std::sqrt((1.0 - x[k]) * (1.0 + x[k]));
  }
  // weights from the unweighted columns
  PlanHost Q;
  Q.l = n;
  Q.row_x = x;
  Q.row_sin = sin_theta;
  Q.row_sqw.assign(n, 1.0);
  std::vector<double> sum(n, 0.0);
  const int rchunks = (n + kChunk - 1) / kChunk;
  parallel_for(rchunks, [&](int ch) {
    const int r0 = ch * kChunk, nr = std::min(n, r0 + kChunk) - r0;
    std::vector<double> col(nr);
    ColumnStream cs(Q, m, p, nr, r0);
    for (int j = 0; j < n; ++j) {
      cs.next(col.data());
      for (int i = 0; i < nr; ++i) sum[r0 + i] += col[i] * col[i];
    }
  });
  rho.resize(n);
  for (int i = 0; i < n; ++i) rho[i] = sum[i] > 0.0 ? 1.0 / sum[i] : 0.0;
}

}  // namespace sht

extern "C" sht_status sht_gauss_jacobi_nodes(int m, int parity, int n, double* x, double* rho) {
  if (!x || !rho || m < 0 || n < 1 || n > SHT_UNIT_STATS_MAX_L || (parity != 0 && parity != 1))
    return SHT_ERR_INVALID_ARG;
  try {
    std::vector<double> xs, th, r;
    sht::gauss_jacobi_nodes(m, parity, n, xs, th, r);
    std::copy(xs.begin(), xs.end(), x);
    std::copy(r.begin(), r.end(), rho);
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (...) {
    return SHT_ERR_INVALID_ARG;
  }
  return SHT_OK;
}

extern "C" sht_status sht_unit_stats_gauss_jacobi(int n, int m, int parity, double eps_id, const sht_plan_opts* opts,
                                                  unsigned long long seed, sht_unit_stats* out) {
  sht_plan_opts o;
  if (!out || n < 1 || n > SHT_UNIT_STATS_MAX_L || m < 0 || (parity != 0 && parity != 1) || !(eps_id > 0.0) ||
      !(eps_id < 1.0) || !options_ok(opts, &o))
    return SHT_ERR_INVALID_ARG;
  try {
    sht::PlanHost P;
    P.l = n;
    P.unit_cols = n;
    apply_options(P, o, eps_id);
    const double t0 = now_s();
    std::vector<double> rho;
    sht::gauss_jacobi_nodes(m, parity, n, P.row_x, P.row_sin, rho);
    P.row_sqw.resize(n);
    for (int i = 0; i < n; ++i) P.row_sqw[i] = std::sqrt(rho[i]);
    return unit_stats_of(P, m, parity, eps_id, now_s() - t0, seed, out);
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (...) {
    return SHT_ERR_INVALID_ARG;
  }
}

extern "C" sht_status sht_unit_stats_compute(int l, int m, int parity, double eps_id, const sht_plan_opts* opts,
                                             unsigned long long seed, sht_unit_stats* out) {
  sht_plan_opts o;
  if (!out || l < 1 || l > SHT_UNIT_STATS_MAX_L || m < 0 || m >= 2 * l || (parity != 0 && parity != 1) ||
      !(eps_id > 0.0) || !(eps_id < 1.0) || !options_ok(opts, &o))
    return SHT_ERR_INVALID_ARG;
  try {
    sht::PlanHost P;
    P.l = l;
    apply_options(P, o, eps_id);
    const double t0 = now_s();
    sht::gl_nodes(2 * l, P.x, P.w, P.sin_pos, P.num_threads);
    return unit_stats_of(P, m, parity, eps_id, now_s() - t0, seed, out);
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (...) {
    return SHT_ERR_INVALID_ARG;
  }
}

extern "C" sht_status sht_interp_decomp(const double* A, int h, int w, double eps, int* k, int* perm, double* T,
                                        int* swaps) {
  if (!A || !k || !perm || !T || h < 1 || w < 1 || w > 65535 || !(eps > 0.0)) return SHT_ERR_INVALID_ARG;
  try {
    std::vector<double> work(A, A + (size_t)h * w);
    std::vector<int> p;
    std::vector<double> t;
    int sw = 0;
    const int kk = sht::interp_decomp(work.data(), h, w, eps, p, t, &sw);
    *k = kk;
    std::copy(p.begin(), p.end(), perm);
    std::copy(t.begin(), t.end(), T);
    if (swaps) *swaps = sw;
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (...) {
    return SHT_ERR_INVALID_ARG;
  }
  return SHT_OK;
}
