// MIMO detection on the Ising solver (supplementary DI-MIMO sections): host-side FP64
// formulation of the residual problem around an MMSE estimate, and reconstruction of the
// detected symbols from spins.  The Ising solving itself runs in the device kernels.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "mimo.h"
#include "pim.h"

namespace pim {

using cd = std::complex<double>;

int mimo_spins_per_component(int qam) {
  if (qam == 4 || qam == 16) return 2;  // corrections {-2, 0, 2}: T = [I, I]
  if (qam == 64) return 3;              // corrections {-4, .., 4}: T = [2I, I, I]
  return 0;
}

int mimo_depth(int qam, int depth) {
  if (mimo_spins_per_component(qam) == 0) return 0;
  if (depth == 0) return mimo_spins_per_component(qam);
  return depth == 2 || depth == 3 ? depth : 0;
}

// Weight of spin block b in T: [I, I] (depth 2) or [2I, I, I] (depth 3).
static double weight_of_block(int depth, int b) { return (depth == 3 && b == 0) ? 2.0 : 1.0; }

static int pam_levels(int qam) { return qam == 4 ? 2 : (qam == 16 ? 4 : 8); }

// Nearest point of {-L+1, -L+3, .., L-1}.
static double slice_pam(double v, int L) {
  double k = std::floor((v + L) / 2.0);
  if (k < 0) k = 0;
  if (k > L - 1) k = L - 1;
  return 2.0 * k - L + 1;
}

// Solves (H^H H + reg I) z = H^H y by a complex Cholesky factorisation (the matrix is
// Hermitian positive definite for reg > 0).  Returns false if a pivot is not positive.
static bool mmse_solve(int nt, int nr, const cd* H, const cd* y, double reg, cd* z,
                       std::vector<cd>& gram) {
  std::vector<cd> A(static_cast<size_t>(nt) * nt), b(nt);
  gram.assign(static_cast<size_t>(nt) * nt, 0.0);
  for (int i = 0; i < nt; ++i) {
    for (int j = i; j < nt; ++j) {  // Hermitian: one triangle
      cd acc = 0;
      for (int r = 0; r < nr; ++r) acc += std::conj(H[r * nt + i]) * H[r * nt + j];
      gram[i * nt + j] = acc;
      gram[j * nt + i] = std::conj(acc);
    }
  }
  for (int i = 0; i < nt; ++i) {
    for (int j = 0; j < nt; ++j) A[i * nt + j] = gram[i * nt + j] + (i == j ? reg : 0.0);
    cd acc = 0;
    for (int r = 0; r < nr; ++r) acc += std::conj(H[r * nt + i]) * y[r];
    b[i] = acc;
  }
  // A = L L^H, L lower triangular
  std::vector<cd> L(static_cast<size_t>(nt) * nt, 0.0);
  for (int j = 0; j < nt; ++j) {
    double d = A[j * nt + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(L[j * nt + k]);
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j * nt + j] = ljj;
    for (int i = j + 1; i < nt; ++i) {
      cd acc = A[i * nt + j];
      for (int k = 0; k < j; ++k) acc -= L[i * nt + k] * std::conj(L[j * nt + k]);
      L[i * nt + j] = acc / ljj;
    }
  }
  std::vector<cd> w(nt);
  for (int i = 0; i < nt; ++i) {  // L w = b
    cd acc = b[i];
    for (int k = 0; k < i; ++k) acc -= L[i * nt + k] * w[k];
    w[i] = acc / L[i * nt + i];
  }
  for (int i = nt - 1; i >= 0; --i) {  // L^H z = w
    cd acc = w[i];
    for (int k = i + 1; k < nt; ++k) acc -= std::conj(L[k * nt + i]) * z[k];
    z[i] = acc / L[i * nt + i].real();
  }
  return true;
}

int mimo_formulate(int nt, int nr, int qam, const double* H_ri, const double* y_ri, double reg,
                   double* J_out, double* h_out, double* xm_ri, int depth) {
  const int ncopy = mimo_depth(qam, depth);
  const int two_nt = 2 * nt, n = ncopy * two_nt;
  const int L = pam_levels(qam);
  std::vector<cd> H(static_cast<size_t>(nr) * nt), y(nr), z(nt), gram;
  for (int k = 0; k < nr * nt; ++k) H[k] = cd(H_ri[2 * k], H_ri[2 * k + 1]);
  for (int k = 0; k < nr; ++k) y[k] = cd(y_ri[2 * k], y_ri[2 * k + 1]);
  if (!mmse_solve(nt, nr, H.data(), y.data(), reg, z.data(), gram)) return PIM_ERR_INVALID;
  std::vector<cd> xm(nt);
  for (int c = 0; c < nt; ++c) {
    xm[c] = cd(slice_pam(z[c].real(), L), slice_pam(z[c].imag(), L));
    xm_ri[2 * c] = xm[c].real();
    xm_ri[2 * c + 1] = xm[c].imag();
  }
  // Real-valued equivalent Hr = [[Re H, -Im H], [Im H, Re H]] without forming it:
  //   Hr^T Hr = [[Re G, -Im G], [Im G, Re G]] with G = H^H H, and
  //   Hr^T [Re rho; Im rho] = [Re(H^H rho); Im(H^H rho)] for the residual rho = y - H x_m.
  std::vector<double> Gr(static_cast<size_t>(two_nt) * two_nt), g(two_nt);
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const cd v = gram[a * nt + b];
      Gr[a * two_nt + b] = v.real();
      Gr[a * two_nt + nt + b] = -v.imag();
      Gr[(nt + a) * two_nt + b] = v.imag();
      Gr[(nt + a) * two_nt + nt + b] = v.real();
    }
  std::vector<cd> rho(nr);
  for (int r = 0; r < nr; ++r) {
    cd acc = y[r];
    for (int c = 0; c < nt; ++c) acc -= H[r * nt + c] * xm[c];
    rho[r] = acc;
  }
  for (int c = 0; c < nt; ++c) {
    cd acc = 0;
    for (int r = 0; r < nr; ++r) acc += std::conj(H[r * nt + c]) * rho[r];
    g[c] = acc.real();
    g[nt + c] = acc.imag();
  }
  const std::vector<double>& G = Gr;
  // spin k = block b * 2nt + component m, T[m][k] = w_b:
  //   J[k][l] = -2 w_b w_c G[m][m'] (k != l),  h[k] = 2 w_b g[m]
  for (int k = 0; k < n; ++k) {
    const int bk = k / two_nt, mk = k % two_nt;
    const double wk = weight_of_block(ncopy, bk);
    for (int l = 0; l < n; ++l) {
      const int bl = l / two_nt, ml = l % two_nt;
      J_out[static_cast<size_t>(k) * n + l] =
          k == l ? 0.0 : -2.0 * wk * weight_of_block(ncopy, bl) * G[mk * two_nt + ml];
    }
    h_out[k] = 2.0 * wk * g[mk];
  }
  return PIM_OK;
}

void mimo_reconstruct(int nt, int qam, const double* xm_ri, const int8_t* spins, double* x_ri,
                      int depth) {
  const int ncopy = mimo_depth(qam, depth), two_nt = 2 * nt, L = pam_levels(qam);
  for (int m = 0; m < two_nt; ++m) {
    double d = 0.0;
    for (int b = 0; b < ncopy; ++b) d += weight_of_block(ncopy, b) * spins[b * two_nt + m];
    const int c = m % nt;
    const double base = m < nt ? xm_ri[2 * c] : xm_ri[2 * c + 1];
    x_ri[2 * c + (m < nt ? 0 : 1)] = slice_pam(base + d, L);
  }
}

}  // namespace pim
