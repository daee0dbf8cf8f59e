// Host-side (FP64) plan construction for the exact exponential field step.
//
// For every azimuthal mode m the discrete operator of Sec. 2.5 (Eqs.
// spatialAM_maxwell_Er ... _Bz) separates, after a DFT along periodic z, into
// two radial families per kz:
//   TM: (E_z, grad part of E_perp, grad part of w)   with w = (B_theta, -B_rho)
//   TE: (curl part of E_perp, curl part of w, B_z)
// Each family is diagonalised by one kz-independent real radial basis
// (eigenvectors of L0 = D_div^(+) D^(-) - m^2/rho^2 on the primary grid and of
// L2 = D_div^(-) D^(+) - m^2/rho_-^2 on the staggered grid), leaving a 3x3 block
// per (kz, j) with eigenvalues {0, +-i omega}, omega^2 = kappa(kz)^2 + lambda_j.
// The radial divergence/curl stencils are folded into dense projection (P) and
// back-projection (Q) matrices; the axis rule of Sec. 2.4 is folded into Q's
// axis rows.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace fdetd {

// Coefficient closed forms (Sec. 2.3): staggered first derivative of order 2N,
// centred first and second derivatives, axis extrapolation of Sec. 2.4.
std::vector<double> staggered_coeffs(int order);
std::vector<double> centred_d1_coeffs(int order);
std::vector<double> centred_d2_coeffs(int order, double* e0);
std::vector<double> axis_coeffs(int N);
// Centred first (d1[0..N-1]) and second (e2[0..N-1], e0) derivative coefficients written into
// caller arrays (no allocation); returns N = order/2 or -1 for an invalid order.
int centred_coeffs_fixed(int order, double* d1, double* e2, double* e0);

// Per-mode radial tables.  All matrices are row-major (3n x 3n), n = Nr.
//  Field blocks (columns of P, rows of Q), E group: (Er, Et^, Ez); B group: (Bt, Br^, Bz^)
//  Coefficient blocks, E group: (e, a, c^); B group: (b, d^, f^).
//  ^ marks the rotated variable tau*F with tau = i*sigma = -i (sigma = -1 mode sign),
//  which makes every radial matrix real.
struct ModePlan {
  int m = 0, n = 0;
  std::vector<double> lam, mu;          // n each; lam = TM eigenvalues, mu = TE (slot n-1 special)
  std::vector<uint8_t> tm_live, te_live;  // 1 where the 3x3 rotation applies, 0 = identity
  std::vector<double> PE, PB, QE, QB;   // (3n)^2 each
  double max_imag = 0.0;                // largest |Im| met in the eigen-solves
};

struct HostPlan {
  int Nz = 0, Nr = 0, order = 0;
  double dz = 0, dr = 0, dt = 0;
  std::vector<int> modes;
  std::vector<ModePlan> mp;
  std::vector<double> sp_re, sp_im, sm_re, sm_im, kappa2;  // z symbols, Nz each
};

// Builds the full host plan.  Returns 0 on success; nonzero with msg set otherwise
// (1 = bad argument, 4 = eigen-solve failure).
int build_host_plan(HostPlan& hp, int Nz, int Nr, const int* modes, int nmodes, int order, double dz,
                    double dr, double dt, std::string& msg);

// Process-wide cache of per-mode radial tables (keyed on Nr, order, dr, m): byte limit (0 empties and disables
// it; default 4 GiB) and counters.
void mode_cache_set_limit(size_t bytes);
// Builds mode m's tables into the cache unless present (0, or 4 with msg for a failed eigen-solve).
int mode_cache_warm(int n, int order, double dr, int m, std::string& msg);
void mode_cache_stats(size_t* bytes, size_t* limit, int* entries, uint64_t* hits, uint64_t* misses);

// Banded radial operators of H for the Taylor scheme (layout documented at the definition).
// Returns 0, or 1 for a bad order / too few radial points.
int taylor_bands(int n, int order, double dr, int m, std::vector<double>& bands, std::vector<double>& axis);

// Banded operators and LU factors of the planar current correction (layout at the definition).
int current_bands(int n, int order, double dr, int m, std::vector<double>& divp, std::vector<double>& dm,
                  std::vector<double>& lo, std::vector<double>& up);

// Phase coefficients of exp(t M) = I + A1 M + A2 M^2 for a 3x3 block with eigenvalues {0, +-i w}:
// A1 = sin(w t)/w, A2 = (1 - cos(w t))/w^2 (limits at w = 0).
void phase_coeffs(double w, double t, double* A1, double* A2);

}  // namespace fdetd
