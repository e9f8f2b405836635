// Host-side FP64 setup of the GB300 MGRIT library: discretisation data and
// the least-squares coarse operators.  Internal interface (not part of the ABI).
#pragma once
#include <complex>
#include <string>
#include <vector>

namespace mg {

using cplx = std::complex<double>;

// (offset, coefficient) taps of a circulant stencil: (T v)_r = sum c v_{r+off}.
struct Taps {
  std::vector<int> off;
  std::vector<double> coef;
  int size() const { return (int)off.size(); }
  int lo() const;   // most negative offset (0 if none below)
  int hi() const;   // most positive offset (0 if none above)
};

// Butcher tableau, A row-major s x s (Appendix A).
struct Tableau {
  int s = 0;
  std::vector<double> A, b;
  double a(int i, int j) const { return A[i * s + j]; }
};

Tableau erk_tableau(int p);
Tableau sdirk_tableau(int p);

// dt*L for U_p at CFL number c (Section 2.1): -(c/s_p) sum_k a_k v_{i+k}.
Taps dtL_taps(int upwind_order, double c);

// Stability function R(z) = 1 + z b^T (I - zA)^{-1} 1 (Lemma 1).
cplx stability(const Tableau& t, cplx z);

// Eigenvalue of a stencil on Fourier mode theta_k = 2 pi k / nx, all k.
std::vector<cplx> stencil_symbol(const Taps& t, int nx);

// In-place DFT (forward: sum_j a_j e^{-2 pi i jk/n}); inverse includes 1/n.
void dft(std::vector<cplx>& a, bool inverse);

// One ERK step as a single stencil (Corollary 1), from the stage form.
Taps erk_phi_taps(int rk_order, int upwind_order, double c);

// T^k as one stencil (repeated convolution of the taps, contiguous offsets
// k*lo .. k*hi), accumulated in long double.
Taps taps_power(const Taps& t, int k);

// A fitted coarse operator and its diagnostics.
struct CoarseOp {
  Taps taps;
  std::vector<cplx> mu;     // eigenvalues
  double imag = 0.0;        // max |Im| of the complex least-squares solution
  double bound = 0.0;       // max_k Eq. 4 over |lambda_k| < 1 at the level's nt
  double mumax = 0.0;       // max_k |mu_k|
};

struct PlanRequest {
  int nx, nt, family, rk_order, upwind_order;
  double cfl;
  int m, levels, rule, halfwidth;
  double eta, rho;
  const int* user_nnz;
  const int* user_off;
  const double* user_coef;
};

// Build Psi_2..Psi_L.  Returns false and sets *err on failure.
bool build_hierarchy(const PlanRequest& rq, std::vector<CoarseOp>* ops, std::string* err);

// Rows of an operator on the non-periodic domain (Section 4.5) that differ
// from its circulant: rows 0..nl-1 over columns 0..cl-1 and rows nx-nr..nx-1
// over columns nx-cr..nx-1, row-major, the left block first.  Every other row
// is the circulant's and never reaches past either end.
struct BoundaryRows {
  int nl = 0, cl = 0, nr = 0, cr = 0;
  std::vector<double> w;
};

// Lagrange weights of degree q through the nodes 0, -1, .., -q evaluated at
// j: the outflow ghost u_{nx-1+j} = sum_k w_k u_{nx-1-k}.
std::vector<double> extrapolation_weights(int q, int j);

// Phi^m of ERKp+Uq with a homogeneous inflow condition at x = -1 (zero
// ghost values left of the domain in every stage) and degree-q
// extrapolation to the outflow ghosts in every stage; nx unknowns
// x_i = -1 + (i+1) dx.  Empty (nl = nr = 0) if nx is too small for the two
// ends to stay apart.
BoundaryRows inflow_phi_rows(int rk_order, int upwind_order, double c, int nx, int m = 1);

// Weighted least-squares fit of Eq. 6 on the given offsets; nt_level sets
// the Eq. 4 bound's horizon.
CoarseOp lsq_fit(const std::vector<cplx>& lam, const std::vector<double>& col_m,
                 const std::vector<int>& offsets, int m, int nt_level, bool unit_weight = false);

// Roots of sum_k p[k] z^k (p.size()-1 >= 1), Aberth iteration + Newton polish.
std::vector<cplx> poly_roots(const std::vector<double>& p);

// ERK CFL limit: largest c with max_theta |R| <= 1 + 1e-6 (Table 1's values).
double erk_cfl_limit(int rk_order, int upwind_order);

}  // namespace mg
