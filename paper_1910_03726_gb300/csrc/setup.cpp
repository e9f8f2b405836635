// Host FP64 setup: U_p stencils and Runge-Kutta tableaux (Section 2.1,
// Appendix A), stability function and Fourier symbols (Lemma 1), the
// collapsed ERK propagator (Corollary 1), and the weighted least-squares
// coarse operators Psi (Eq. 6, Sections 4.1-4.6) with the two-level bound
// (Eq. 4).  Runs once per handle; not on the timed path.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace mg {

static const double kPi = 3.14159265358979323846264338327950288;
static const double kEpsWeight = 1e-6;   // weight-function epsilon, Section 4
static const double kImagFlag = 1e-8;    // fit acceptance limit, Section 4.1

int Taps::lo() const {
  int v = 0;
  for (int o : off) v = std::min(v, o);
  return v;
}
int Taps::hi() const {
  int v = 0;
  for (int o : off) v = std::max(v, o);
  return v;
}

// ---------------------------------------------------------------- tableaux

Tableau erk_tableau(int p) {
  Tableau t;
  switch (p) {
    case 1: t.s = 1; t.A = {0.0}; t.b = {1.0}; break;
    case 2: t.s = 2; t.A = {0, 0, 1, 0}; t.b = {0.5, 0.5}; break;
    case 3:
      t.s = 3;
      t.A = {0, 0, 0, 1, 0, 0, 0.25, 0.25, 0};
      t.b = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
      break;
    case 4:
      t.s = 4;
      t.A = {0, 0, 0, 0, 0.5, 0, 0, 0, 0, 0.5, 0, 0, 0, 0, 1, 0};
      t.b = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
      break;
    case 5:  // six stages, Butcher's fifth-order method
      t.s = 6;
      t.A.assign(36, 0.0);
      t.A[1 * 6 + 0] = 0.25;
      t.A[2 * 6 + 0] = 0.125; t.A[2 * 6 + 1] = 0.125;
      t.A[3 * 6 + 2] = 0.5;
      t.A[4 * 6 + 0] = 3.0 / 16.0; t.A[4 * 6 + 1] = -3.0 / 8.0;
      t.A[4 * 6 + 2] = 3.0 / 8.0; t.A[4 * 6 + 3] = 9.0 / 16.0;
      t.A[5 * 6 + 0] = -3.0 / 7.0; t.A[5 * 6 + 1] = 8.0 / 7.0; t.A[5 * 6 + 2] = 6.0 / 7.0;
      t.A[5 * 6 + 3] = -12.0 / 7.0; t.A[5 * 6 + 4] = 8.0 / 7.0;
      t.b = {7.0 / 90.0, 0.0, 32.0 / 90.0, 12.0 / 90.0, 32.0 / 90.0, 7.0 / 90.0};
      break;
    default: t.s = 0;
  }
  return t;
}

Tableau sdirk_tableau(int p) {
  Tableau t;
  switch (p) {
    case 1: t.s = 1; t.A = {1.0}; t.b = {1.0}; break;
    case 2: {
      double g = 1.0 - std::sqrt(2.0) / 2.0, h = std::sqrt(2.0) / 2.0;
      t.s = 2; t.A = {g, 0.0, h, g}; t.b = {h, g};
      break;
    }
    case 3: {
      const double z = 0.43586652150845899942;  // root of x^3 - 3x^2 + 3x/2 - 1/6
      double beta = (1.0 - z) / 2.0;
      double gam = -1.5 * z * z + 4.0 * z - 0.25;
      double eps = 1.5 * z * z - 5.0 * z + 1.25;
      t.s = 3;
      t.A = {z, 0, 0, beta, z, 0, gam, eps, z};
      t.b = {gam, eps, z};
      break;
    }
    case 4: {
      t.s = 5;
      t.A.assign(25, 0.0);
      for (int i = 0; i < 5; ++i) t.A[i * 5 + i] = 0.25;
      t.A[1 * 5 + 0] = 0.5;
      t.A[2 * 5 + 0] = 17.0 / 50.0; t.A[2 * 5 + 1] = -1.0 / 25.0;
      t.A[3 * 5 + 0] = 371.0 / 1360.0; t.A[3 * 5 + 1] = -137.0 / 2720.0; t.A[3 * 5 + 2] = 15.0 / 544.0;
      t.A[4 * 5 + 0] = 25.0 / 24.0; t.A[4 * 5 + 1] = -49.0 / 48.0; t.A[4 * 5 + 2] = 125.0 / 16.0;
      t.A[4 * 5 + 3] = -85.0 / 12.0;
      t.b.assign(t.A.begin() + 20, t.A.begin() + 25);
      break;
    }
    default: t.s = 0;
  }
  return t;
}

// ------------------------------------------------------------------ stencils

Taps dtL_taps(int q, double c) {
  // v'_i ~ (1/(s dx)) sum_k a_k v_{i+k}; L = -alpha d/dx, so dt L has -c a_k / s.
  static const int S[6] = {0, 1, 2, 6, 12, 60};
  static const int K[6][6] = {{0}, {-1, 0}, {-2, -1, 0}, {-2, -1, 0, 1}, {-3, -2, -1, 0, 1}, {-3, -2, -1, 0, 1, 2}};
  static const int A[6][6] = {{0}, {-1, 1}, {1, -4, 3}, {1, -6, 3, 2}, {-1, 6, -18, 10, 3}, {-2, 15, -60, 20, 30, -3}};
  Taps t;
  if (q < 1 || q > 5) return t;
  for (int j = 0; j <= q; ++j) {
    t.off.push_back(K[q][j]);
    t.coef.push_back(-c * (double)A[q][j] / (double)S[q]);
  }
  return t;
}

cplx stability(const Tableau& t, cplx z) {
  // (I - zA) y = 1 by forward substitution (A is lower triangular here).
  std::vector<cplx> y(t.s);
  cplx acc = 0.0;
  for (int i = 0; i < t.s; ++i) {
    cplx r = 1.0;
    for (int j = 0; j < i; ++j) r += z * t.a(i, j) * y[j];
    y[i] = r / (1.0 - z * t.a(i, i));
    acc += t.b[i] * y[i];
  }
  return 1.0 + z * acc;
}

std::vector<cplx> stencil_symbol(const Taps& t, int nx) {
  std::vector<cplx> out(nx);
  for (int k = 0; k < nx; ++k) {
    cplx s = 0.0;
    for (int j = 0; j < t.size(); ++j) {
      long long e = ((long long)t.off[j] * k) % nx;
      if (e < 0) e += nx;
      double ang = 2.0 * kPi * (double)e / (double)nx;
      s += t.coef[j] * cplx(std::cos(ang), std::sin(ang));
    }
    out[k] = s;
  }
  return out;
}

void dft(std::vector<cplx>& a, bool inverse) {
  const int n = (int)a.size();
  if (n <= 1) return;
  const double sgn = inverse ? 1.0 : -1.0;
  if ((n & (n - 1)) == 0) {
    // iterative radix-2 Cooley-Tukey: bit reversal, then butterflies
    for (int i = 1, j = 0; i < n; ++i) {
      int bit = n >> 1;
      for (; j & bit; bit >>= 1) j ^= bit;
      j ^= bit;
      if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<cplx> w(n / 2);
    for (int k = 0; k < n / 2; ++k) {
      double ang = sgn * 2.0 * kPi * (double)k / (double)n;
      w[k] = cplx(std::cos(ang), std::sin(ang));
    }
    for (int len = 2; len <= n; len <<= 1) {
      int step = n / len;
      for (int i = 0; i < n; i += len)
        for (int k = 0; k < len / 2; ++k) {
          cplx u = a[i + k], v = a[i + k + len / 2] * w[k * step];
          a[i + k] = u + v;
          a[i + k + len / 2] = u - v;
        }
    }
  } else {
    std::vector<cplx> out(n);
    for (int k = 0; k < n; ++k) {
      cplx s = 0.0;
      for (int j = 0; j < n; ++j) {
        long long e = ((long long)j * k) % n;
        double ang = sgn * 2.0 * kPi * (double)e / (double)n;
        s += a[j] * cplx(std::cos(ang), std::sin(ang));
      }
      out[k] = s;
    }
    a.swap(out);
  }
  if (inverse)
    for (auto& v : a) v /= (double)n;
}

// Apply taps on an open line (no wrap); `v` indexed from -S..S via base S.
static std::vector<double> apply_line(const Taps& t, const std::vector<double>& v, int S) {
  std::vector<double> out(v.size(), 0.0);
  for (int x = -S; x <= S; ++x) {
    double acc = 0.0;
    for (int j = 0; j < t.size(); ++j) {
      int y = x + t.off[j];
      if (y >= -S && y <= S) acc += t.coef[j] * v[y + S];
    }
    out[x + S] = acc;
  }
  return out;
}

Taps erk_phi_taps(int rk_order, int upwind_order, double c) {
  Tableau tb = erk_tableau(rk_order);
  Taps L = dtL_taps(upwind_order, c);
  Taps out;
  if (tb.s == 0 || L.size() == 0) return out;
  int reach = std::max(-L.lo(), L.hi());
  int S = tb.s * reach + 1;
  std::vector<double> u(2 * S + 1, 0.0);
  u[S] = 1.0;  // e_0
  std::vector<std::vector<double>> K;
  for (int i = 0; i < tb.s; ++i) {
    std::vector<double> y = u;
    for (int j = 0; j < i; ++j)
      if (tb.a(i, j) != 0.0)
        for (size_t x = 0; x < y.size(); ++x) y[x] += tb.a(i, j) * K[j][x];
    K.push_back(apply_line(L, y, S));
  }
  std::vector<double> r = u;
  for (int i = 0; i < tb.s; ++i)
    if (tb.b[i] != 0.0)
      for (size_t x = 0; x < r.size(); ++x) r[x] += tb.b[i] * K[i][x];
  // r = Phi e_0 = first column; offset i carries column entry at row -i
  for (int i = -S; i <= S; ++i) {
    double v = r[-i + S];
    if (v != 0.0) {
      out.off.push_back(i);
      out.coef.push_back(v);
    }
  }
  return out;
}

std::vector<double> extrapolation_weights(int q, int j) {
  std::vector<double> w(q + 1, 1.0);
  for (int k = 0; k <= q; ++k)
    for (int r = 0; r <= q; ++r)
      if (r != k) w[k] *= (double)(j + r) / (double)(r - k);  // nodes -k, -r
  return w;
}

// One stage-wise ERK step of the closed problem on np unknowns (inflow
// ghosts zero, outflow ghosts extrapolated from every stage's input).
static std::vector<double> inflow_step(const Tableau& tb, const Taps& L, int q, const std::vector<double>& u) {
  const int np = (int)u.size(), lo = L.lo(), hi = L.hi();
  std::vector<std::vector<double>> ew;
  for (int j = 1; j <= hi; ++j) ew.push_back(extrapolation_weights(q, j));
  auto dtl = [&](const std::vector<double>& y) {
    std::vector<double> ext(np - lo + hi, 0.0);  // [-lo zeros | y | hi ghosts]
    for (int i = 0; i < np; ++i) ext[i - lo] = y[i];
    for (int j = 1; j <= hi; ++j) {
      double g = 0.0;
      for (int k = 0; k <= q; ++k) g += ew[j - 1][k] * y[np - 1 - k];
      ext[np - 1 + j - lo] = g;
    }
    std::vector<double> out(np, 0.0);
    for (int i = 0; i < np; ++i)
      for (int k = 0; k < L.size(); ++k) out[i] += L.coef[k] * ext[i + L.off[k] - lo];
    return out;
  };
  std::vector<std::vector<double>> K;
  for (int i = 0; i < tb.s; ++i) {
    std::vector<double> y = u;
    for (int j = 0; j < i; ++j)
      if (tb.a(i, j) != 0.0)
        for (int x = 0; x < np; ++x) y[x] += tb.a(i, j) * K[j][x];
    K.push_back(dtl(y));
  }
  std::vector<double> r = u;
  for (int i = 0; i < tb.s; ++i)
    if (tb.b[i] != 0.0)
      for (int x = 0; x < np; ++x) r[x] += tb.b[i] * K[i][x];
  return r;
}

BoundaryRows inflow_phi_rows(int rk_order, int upwind_order, double c, int nx, int m) {
  BoundaryRows B;
  const Tableau tb = erk_tableau(rk_order);
  const Taps L = dtL_taps(upwind_order, c);
  if (tb.s == 0 || L.size() == 0 || m < 1) return B;
  const int s = tb.s, lo = L.lo(), hi = L.hi(), q = upwind_order;
  // rows of Phi^m whose m steps reach a ghost value: the rows that wrap in
  // the circulant Phi^m
  const int nl = m * s * -lo, nr = m * s * hi;
  // the two ends stay apart (one step's closures)
  if (nx < 2 * s * (hi - lo) + q + 2 || nl + nr > nx) return B;
  // The blocks do not depend on nx once the m-step domains of dependence of
  // the two blocks cannot meet: probe a short domain np (the whole domain
  // when nx is shorter).
  const int reach = m * (s * (hi - lo) + q + 1);
  const int np = std::min(nx, std::max(64, nl + nr + 2 * reach + 64));
  // Phi on np unknowns by columns, kept as row lists
  std::vector<std::vector<std::pair<int, double>>> rows(np);
  std::vector<double> e(np, 0.0);
  for (int col = 0; col < np; ++col) {
    e[col] = 1.0;
    const std::vector<double> v = inflow_step(tb, L, q, e);
    e[col] = 0.0;
    for (int row = 0; row < np; ++row)
      if (v[row] != 0.0) rows[row].push_back({col, v[row]});
  }
  // boundary row i of Phi^m = e_i^T Phi^m, by m row-vector products
  auto power_row = [&](int i) {
    std::vector<double> v(np, 0.0), w(np);
    v[i] = 1.0;
    for (int k = 0; k < m; ++k) {
      std::fill(w.begin(), w.end(), 0.0);
      for (int r = 0; r < np; ++r)
        if (v[r] != 0.0)
          for (const auto& cv : rows[r]) w[cv.first] += v[r] * cv.second;
      v.swap(w);
    }
    return v;
  };
  std::vector<std::vector<double>> left, right;
  for (int i = 0; i < nl; ++i) left.push_back(power_row(i));
  for (int i = np - nr; i < np; ++i) right.push_back(power_row(i));
  int cl = 0, cmin = np;
  for (const auto& v : left)
    for (int col = 0; col < np; ++col)
      if (v[col] != 0.0) cl = std::max(cl, col + 1);
  for (const auto& v : right)
    for (int col = 0; col < np; ++col)
      if (v[col] != 0.0) cmin = std::min(cmin, col);
  const int cr = nr ? np - cmin : 0;
  B.nl = nl; B.cl = cl; B.nr = nr; B.cr = cr;
  for (const auto& v : left) B.w.insert(B.w.end(), v.begin(), v.begin() + cl);
  for (const auto& v : right) B.w.insert(B.w.end(), v.end() - cr, v.end());
  return B;
}

Taps taps_power(const Taps& t, int k) {
  Taps out;
  if (t.size() == 0 || k < 1) return out;
  const int lo = t.lo(), hi = t.hi();
  std::vector<long double> base(hi - lo + 1, 0.0L), acc(1, 1.0L);
  for (int j = 0; j < t.size(); ++j) base[t.off[j] - lo] += t.coef[j];
  for (int step = 0; step < k; ++step) {  // acc <- acc * base (offsets add)
    std::vector<long double> nxt(acc.size() + base.size() - 1, 0.0L);
    for (size_t a = 0; a < acc.size(); ++a)
      for (size_t b = 0; b < base.size(); ++b) nxt[a + b] += acc[a] * base[b];
    acc.swap(nxt);
  }
  for (size_t a = 0; a < acc.size(); ++a) {
    out.off.push_back(k * lo + (int)a);
    out.coef.push_back((double)acc[a]);
  }
  return out;
}

// Periodic application of taps to a length-nx vector.
static std::vector<double> apply_periodic(const Taps& t, const std::vector<double>& v) {
  int nx = (int)v.size();
  std::vector<double> out(nx, 0.0);
  for (int j = 0; j < t.size(); ++j) {
    int o = ((t.off[j] % nx) + nx) % nx;
    for (int i = 0; i < nx; ++i) {
      int k = i + o;
      if (k >= nx) k -= nx;
      out[i] += t.coef[j] * v[k];
    }
  }
  return out;
}

static std::vector<double> power_column(const Taps& t, int nx, int m) {
  std::vector<double> e(nx, 0.0);
  e[0] = 1.0;
  for (int k = 0; k < m; ++k) e = apply_periodic(t, e);
  return e;
}

static cplx ipow(cplx z, int m) {
  cplx r = 1.0;
  while (m > 0) {
    if (m & 1) r *= z;
    z *= z;
    m >>= 1;
  }
  return r;
}

// ------------------------------------------------------------ least squares

// Diagonal i <-> first-column row (-i) mod nx, i in (-nx/2, nx/2].
static inline double diag_value(const std::vector<double>& col, int i) {
  int nx = (int)col.size();
  int r = ((-i) % nx + nx) % nx;
  return col[r];
}

static double max_bound(const std::vector<cplx>& lam, const std::vector<cplx>& mu, int m, int nt) {
  const int N = nt / m;
  double best = 0.0;
  for (size_t k = 0; k < lam.size(); ++k) {
    double al = std::abs(lam[k]);
    if (!(al < 1.0 - 1e-14)) continue;
    double a = std::pow(al, m) * std::abs(ipow(lam[k], m) - mu[k]);
    double am = std::abs(mu[k]);
    double g = (std::fabs(1.0 - am) > 1e-8) ? (1.0 - std::pow(am, N - 1)) / (1.0 - am) : (double)(N - 1);
    best = std::max(best, std::sqrt((double)m) * a * g);
  }
  return best;
}

CoarseOp lsq_fit(const std::vector<cplx>& lam, const std::vector<double>& col_m,
                 const std::vector<int>& offsets, int m, int nt_level, bool unit_weight) {
  const int n = (int)lam.size(), p = (int)offsets.size();
  CoarseOp op;
  // right-hand side: eigenvalues of the ideal operator = DFT of phi~^m
  std::vector<cplx> rhs(col_m.begin(), col_m.end());
  dft(rhs, false);
  // rows sorted by decreasing weight (Householder QR is then accurate for
  // strongly row-weighted problems); the solution does not depend on order
  std::vector<double> sw(n);
  for (int k = 0; k < n; ++k)
    sw[k] = unit_weight ? 1.0 : 1.0 / std::fabs(1.0 - std::abs(lam[k]) + kEpsWeight);
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sw[a] > sw[b]; });
  std::vector<cplx> A((size_t)n * p), b(n);   // column-major
  for (int r = 0; r < n; ++r) {
    int k = order[r];
    for (int j = 0; j < p; ++j) {
      long long e = ((long long)offsets[j] * k) % n;
      if (e < 0) e += n;
      double ang = 2.0 * kPi * (double)e / (double)n;  // F e_{(-i) mod n} = e^{+2 pi i i k/n}
      A[(size_t)j * n + r] = sw[k] * cplx(std::cos(ang), std::sin(ang));
    }
    b[r] = sw[k] * rhs[k];
  }
  std::vector<cplx> v(n);
  for (int k = 0; k < p; ++k) {
    double nrm2 = 0.0;
    for (int i = k; i < n; ++i) nrm2 += std::norm(A[(size_t)k * n + i]);
    double nrm = std::sqrt(nrm2);
    cplx x0 = A[(size_t)k * n + k];
    cplx phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    cplx alpha = -phase * nrm;
    for (int i = k; i < n; ++i) v[i] = A[(size_t)k * n + i];
    v[k] -= alpha;
    double vn2 = 0.0;
    for (int i = k; i < n; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0.0) continue;
    for (int j = k; j < p; ++j) {
      cplx s = 0.0;
      for (int i = k; i < n; ++i) s += std::conj(v[i]) * A[(size_t)j * n + i];
      s *= 2.0 / vn2;
      for (int i = k; i < n; ++i) A[(size_t)j * n + i] -= s * v[i];
    }
    cplx s = 0.0;
    for (int i = k; i < n; ++i) s += std::conj(v[i]) * b[i];
    s *= 2.0 / vn2;
    for (int i = k; i < n; ++i) b[i] -= s * v[i];
  }
  std::vector<cplx> x(p);
  for (int k = p - 1; k >= 0; --k) {
    cplx s = b[k];
    for (int j = k + 1; j < p; ++j) s -= A[(size_t)j * n + k] * x[j];
    x[k] = s / A[(size_t)k * n + k];
  }
  op.imag = 0.0;
  for (int j = 0; j < p; ++j) {
    op.taps.off.push_back(offsets[j]);
    op.taps.coef.push_back(x[j].real());     // Lemma 2: the solution is real
    op.imag = std::max(op.imag, std::fabs(x[j].imag()));
  }
  // eigenvalues of the fitted circulant and diagnostics
  std::vector<cplx> col(n, 0.0);
  for (int j = 0; j < p; ++j) {
    int r = ((-offsets[j]) % n + n) % n;
    col[r] += op.taps.coef[j];
  }
  dft(col, false);
  op.mu = col;
  op.mumax = 0.0;
  for (auto& z : op.mu) op.mumax = std::max(op.mumax, std::abs(z));
  op.bound = max_bound(lam, op.mu, m, nt_level);
  return op;
}

// ----------------------------------------------------------------- patterns

static int argmax_offset(const std::vector<double>& col) {
  int nx = (int)col.size();
  int best_i = 0;
  double best_v = -1.0;
  int best_a = 0;
  for (int i = -(nx / 2) + 1; i <= nx / 2; ++i) {
    double v = std::fabs(diag_value(col, i));
    int a = std::abs(i);
    if (v > best_v || (v == best_v && a < best_a)) {
      best_v = v; best_i = i; best_a = a;
    }
  }
  return best_i;
}

static std::vector<int> best_window(const std::vector<double>& col, int width) {
  int nx = (int)col.size();
  int lo = -(nx / 2) + 1;
  double best = -1.0;
  int best_start = lo;
  for (int start = lo; start <= nx / 2 + 1 - width; ++start) {
    double e = 0.0;
    for (int i = start; i < start + width; ++i) {
      double d = diag_value(col, i);
      e += d * d;
    }
    if (e > best * (1.0 + 1e-13)) {
      best = e;
      best_start = start;
    }
  }
  std::vector<int> w;
  for (int i = 0; i < width; ++i) w.push_back(best_start + i);
  return w;
}

static std::vector<int> threshold_pattern(const std::vector<double>& col, double eta) {
  int nx = (int)col.size();
  double mx = 0.0;
  for (int i = -(nx / 2) + 1; i <= nx / 2; ++i) mx = std::max(mx, std::fabs(diag_value(col, i)));
  std::vector<int> out;
  for (int i = -(nx / 2) + 1; i <= nx / 2; ++i)
    if (std::fabs(diag_value(col, i)) >= eta * mx) out.push_back(i);
  return out;
}

static double eta_table(int p, int m) {
  // eta_tol per (p, m) for SDIRKp+Up, Section 4.6
  static const double T[5][6] = {{0},
                                 {.1, .125, .25, .5, .5, .6},
                                 {.05, .1, .1, .2, .2, .2},
                                 {.005, .01, .02, .02, .02, .04},
                                 {.005, .01, .01, .01, .02, .02}};
  int idx = -1;
  for (int k = 0, mm = 2; k < 6; ++k, mm *= 2)
    if (mm == m) idx = k;
  if (p < 1 || p > 4 || idx < 0) return -1.0;
  return T[p][idx];
}

double erk_cfl_limit(int rk_order, int upwind_order) {
  Tableau tb = erk_tableau(rk_order);
  auto maxamp = [&](double c) {
    Taps L = dtL_taps(upwind_order, c);
    double mx = 0.0;
    const int nth = 2048;
    for (int k = 0; k <= nth; ++k) {
      double th = kPi * (double)k / nth;
      cplx z = 0.0;
      for (int j = 0; j < L.size(); ++j) z += L.coef[j] * cplx(std::cos(L.off[j] * th), std::sin(L.off[j] * th));
      mx = std::max(mx, std::abs(stability(tb, z)));
    }
    return mx;
  };
  double lo = 0.0, hi = 3.0;
  for (int it = 0; it < 50; ++it) {
    double mid = 0.5 * (lo + hi);
    if (maxamp(mid) <= 1.0 + 1e-6) lo = mid; else hi = mid;
  }
  return lo;
}

static CoarseOp auto_width(const std::vector<cplx>& lam, const std::vector<double>& col, int m, int nt,
                           int w0, double rho) {
  int nx = (int)lam.size();
  int wmax = std::min(nx - 1, 8 * w0 + 64);
  CoarseOp last;
  for (int W = w0; W <= wmax; ++W) {
    last = lsq_fit(lam, col, best_window(col, W), m, nt);
    if (last.imag <= kImagFlag && last.mumax <= 1.0 + 1e-12 && last.bound <= rho) return last;
  }
  return last;
}

bool build_hierarchy(const PlanRequest& rq, std::vector<CoarseOp>* ops, std::string* err) {
  ops->clear();
  const int nx = rq.nx;
  const bool erk = rq.family == 0;
  Tableau tb = erk ? erk_tableau(rq.rk_order) : sdirk_tableau(rq.rk_order);
  Taps L = dtL_taps(rq.upwind_order, rq.cfl);
  std::vector<cplx> z = stencil_symbol(L, nx), lam(nx);
  for (int k = 0; k < nx; ++k) lam[k] = stability(tb, z[k]);
  Taps phi;
  int nnz_fine = 0;
  if (erk) {
    phi = erk_phi_taps(rq.rk_order, rq.upwind_order, rq.cfl);
    nnz_fine = phi.size();
  }
  std::vector<cplx> cur_lam = lam;
  const Taps* cur = erk ? &phi : nullptr;
  int user_pos = 0;
  for (int lvl = 1; lvl < rq.levels; ++lvl) {
    long long div = 1;
    for (int k = 1; k < lvl; ++k) div *= rq.m;
    int nt_l = (int)(rq.nt / div);
    std::vector<double> col;
    if (cur) {
      col = power_column(*cur, nx, rq.m);
    } else {  // SDIRK fine level: inverse DFT of lambda^m (Section 4.6)
      std::vector<cplx> a(nx);
      for (int k = 0; k < nx; ++k) a[k] = ipow(lam[k], rq.m);
      dft(a, true);
      col.resize(nx);
      for (int k = 0; k < nx; ++k) col[k] = a[k].real();
    }
    CoarseOp op;
    switch (rq.rule) {
      case 1:  // half-width around the argmax
      {
        int i0 = argmax_offset(col);
        std::vector<int> offs;
        for (int i = i0 - rq.halfwidth; i <= i0 + rq.halfwidth; ++i) offs.push_back(i);
        op = lsq_fit(cur_lam, col, offs, rq.m, nt_l);
        break;
      }
      case 0:  // auto: ERK grows a window; SDIRK thresholds with eta_tol(p, m)
      case 2: {
        if (rq.rule == 0 && erk) {
          int w0 = (lvl == 1) ? nnz_fine : ops->back().taps.size();
          op = auto_width(cur_lam, col, rq.m, nt_l, w0, rq.rho);
          break;
        }
        double eta = rq.eta > 0.0 ? rq.eta : eta_table(rq.rk_order, rq.m);
        if (eta <= 0.0) {
          *err = "no eta_tol for this (order, m); pass psi_eta";
          return false;
        }
        op = lsq_fit(cur_lam, col, threshold_pattern(col, eta), rq.m, nt_l);
        break;
      }
      case 3: {  // user supplied
        if (!rq.user_nnz || !rq.user_off || !rq.user_coef) {
          *err = "PSI_USER needs psi_user_nnz/offsets/coeffs";
          return false;
        }
        int n = rq.user_nnz[lvl - 1];
        for (int j = 0; j < n; ++j) {
          op.taps.off.push_back(rq.user_off[user_pos + j]);
          op.taps.coef.push_back(rq.user_coef[user_pos + j]);
        }
        user_pos += n;
        std::vector<cplx> c2(nx, 0.0);
        for (int j = 0; j < n; ++j) c2[((-op.taps.off[j]) % nx + nx) % nx] += op.taps.coef[j];
        dft(c2, false);
        op.mu = c2;
        for (auto& v : op.mu) op.mumax = std::max(op.mumax, std::abs(v));
        op.bound = max_bound(cur_lam, op.mu, rq.m, nt_l);
        break;
      }
      case 4: {  // ideal: all nonzero diagonals of Phi^m
        for (int i = -(nx / 2) + 1; i <= nx / 2; ++i) {
          double v = diag_value(col, i);
          if (v != 0.0) {
            op.taps.off.push_back(i);
            op.taps.coef.push_back(v);
          }
        }
        std::vector<cplx> c2(col.begin(), col.end());
        dft(c2, false);
        op.mu = c2;
        for (auto& v : op.mu) op.mumax = std::max(op.mumax, std::abs(v));
        break;
      }
      default:
        *err = "unknown psi_rule";
        return false;
    }
    if (op.taps.size() == 0) {
      *err = "empty coarse operator";
      return false;
    }
    ops->push_back(op);
    cur_lam = ops->back().mu;
    cur = &ops->back().taps;
  }
  return true;
}

// ---------------------------------------------------------- polynomial roots

std::vector<cplx> poly_roots(const std::vector<double>& pin) {
  std::vector<double> p = pin;
  while (p.size() > 1 && p.back() == 0.0) p.pop_back();
  int d = (int)p.size() - 1;
  std::vector<cplx> z(std::max(d, 0));
  if (d < 1) return z;
  // monic coefficients
  std::vector<cplx> a(d + 1);
  for (int k = 0; k <= d; ++k) a[k] = p[k] / p[d];
  double R = 0.0;
  for (int k = 0; k < d; ++k) R = std::max(R, std::abs(a[k]));
  R = 1.0 + R;  // Cauchy bound
  for (int k = 0; k < d; ++k) {
    double ang = 2.0 * kPi * (k + 0.25) / d + 0.4;
    z[k] = 0.5 * R * cplx(std::cos(ang), std::sin(ang));
  }
  auto eval = [&](cplx x, cplx* dp) {
    cplx v = a[d], dv = 0.0;
    for (int k = d - 1; k >= 0; --k) {
      dv = dv * x + v;
      v = v * x + a[k];
    }
    *dp = dv;
    return v;
  };
  for (int it = 0; it < 500; ++it) {
    double mx = 0.0;
    for (int k = 0; k < d; ++k) {
      cplx dp, v = eval(z[k], &dp);
      if (v == cplx(0.0, 0.0)) continue;
      cplx ratio = v / dp, s = 0.0;
      for (int j = 0; j < d; ++j)
        if (j != k) s += 1.0 / (z[k] - z[j]);
      cplx w = ratio / (1.0 - ratio * s);
      z[k] -= w;
      mx = std::max(mx, std::abs(w) / std::max(1.0, std::abs(z[k])));
    }
    if (mx < 1e-16) break;
  }
  for (int k = 0; k < d; ++k)
    for (int it = 0; it < 3; ++it) {
      cplx dp, v = eval(z[k], &dp);
      if (std::abs(dp) > 0.0) z[k] -= v / dp;
    }
  return z;
}

}  // namespace mg
