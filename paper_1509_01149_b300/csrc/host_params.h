// Host-side checks and factorisations of a controller's constants, shared by every entry
// point that takes (dt, nu, lambda, Sigma, R): mppi_create, mppi_step_static and the
// server's admission.  One copy, so the three accept the same inputs and derive the same
// float constants bit for bit (the same R = lambda Sigma^-1, the same sqrt(nu) chol(Sigma)).
//
//   sampling   du = sqrt(nu) chol(Sigma) eps: Theorem 1 with A = sqrt(nu) I (Sec. III-C);
//              Sigma symmetric positive semi-definite.
//   cost       R symmetric positive definite, or R = lambda Sigma^-1 when none is given (the
//              noise/cost relation of Sec. II), which then needs Sigma positive definite.
#pragma once
#include <cmath>
#include <utility>

namespace mppi {
namespace host {

constexpr int kHostMaxM = 4;

// Textbook Cholesky of a symmetric positive semi-definite m x m matrix (double); false when
// a pivot is negative beyond rounding.
inline bool cholesky_psd(const double *S, int m, double *L) {
  for (int i = 0; i < m * m; ++i) L[i] = 0.0;
  for (int j = 0; j < m; ++j) {
    double d = S[j * m + j];
    for (int l = 0; l < j; ++l) d -= L[j * m + l] * L[j * m + l];
    if (d < -1e-9 * std::fmax(1.0, std::fabs(S[j * m + j]))) return false;
    L[j * m + j] = std::sqrt(std::fmax(d, 0.0));
    for (int i = j + 1; i < m; ++i) {
      double a = S[i * m + j];
      for (int l = 0; l < j; ++l) a -= L[i * m + l] * L[j * m + l];
      L[i * m + j] = L[j * m + j] > 0.0 ? a / L[j * m + j] : 0.0;
    }
  }
  return true;
}

inline bool all_finite(const double *A, int count) {
  for (int i = 0; i < count; ++i)
    if (!std::isfinite(A[i])) return false;
  return true;
}

inline bool symmetric(const double *A, int m) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(A[i * m + j] - A[j * m + i]) > 1e-6 * (std::fabs(A[i * m + j]) + std::fabs(A[j * m + i]) + 1e-30))
        return false;
  return true;
}

// Gauss-Jordan inverse with partial pivoting (double); false if singular.
inline bool invert(const double *A, int m, double *Ai) {
  double a[kHostMaxM * 2 * kHostMaxM];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) a[i * 2 * m + j] = j < m ? A[i * m + j] : (j - m == i ? 1.0 : 0.0);
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(a[r * 2 * m + c]) > std::fabs(a[piv * 2 * m + c])) piv = r;
    if (std::fabs(a[piv * 2 * m + c]) < 1e-300) return false;
    for (int j = 0; j < 2 * m; ++j) std::swap(a[c * 2 * m + j], a[piv * 2 * m + j]);
    const double d = a[c * 2 * m + c];
    for (int j = 0; j < 2 * m; ++j) a[c * 2 * m + j] /= d;
    for (int r = 0; r < m; ++r)
      if (r != c) {
        const double f = a[r * 2 * m + c];
        for (int j = 0; j < 2 * m; ++j) a[r * 2 * m + j] -= f * a[c * 2 * m + j];
      }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Ai[i * m + j] = a[i * 2 * m + m + j];
  return true;
}

// Checks (dt, nu, lambda, Sigma [m][m], R [m][m] or null) and, on success, writes the
// float constants the kernels use: Lnu = sqrt(nu) chol(Sigma) and R (given, or lambda
// Sigma^-1).  Returns null on success, else the reason (a static string).
inline const char *control_constants(int m, float dt, float nu, float lambda, const float *Sigma, const float *R,
                                     float *Lnu, float *R_out) {
  if (m < 1 || m > kHostMaxM) return "control dimension out of range";
  if (!(dt > 0.0f) || !std::isfinite(dt)) return "dt must be finite and > 0";
  if (!(nu > 0.0f) || !std::isfinite(nu)) return "nu must be finite and > 0";
  if (!(lambda > 0.0f) || !std::isfinite(lambda)) return "lambda must be finite and > 0";
  if (!Sigma) return "Sigma is NULL";
  double S[kHostMaxM * kHostMaxM], L[kHostMaxM * kHostMaxM], Rd[kHostMaxM * kHostMaxM];
  for (int i = 0; i < m * m; ++i) S[i] = Sigma[i];
  if (!all_finite(S, m * m)) return "Sigma has a non-finite entry";
  if (!symmetric(S, m)) return "Sigma is not symmetric";
  if (!cholesky_psd(S, m, L)) return "Sigma is not positive semi-definite";
  if (R) {
    for (int i = 0; i < m * m; ++i) Rd[i] = R[i];
    double LR[kHostMaxM * kHostMaxM];
    if (!all_finite(Rd, m * m)) return "R has a non-finite entry";
    if (!symmetric(Rd, m)) return "R is not symmetric";
    if (!cholesky_psd(Rd, m, LR)) return "R is not positive definite";
    for (int j = 0; j < m; ++j)
      if (!(LR[j * m + j] > 0.0)) return "R is not positive definite";
  } else {
    double Si[kHostMaxM * kHostMaxM];
    for (int j = 0; j < m; ++j)
      if (!(L[j * m + j] > 0.0)) return "R = lambda Sigma^-1 needs Sigma positive definite";
    if (!invert(S, m, Si)) return "R = lambda Sigma^-1 needs Sigma positive definite";
    for (int i = 0; i < m * m; ++i) Rd[i] = lambda * Si[i];
  }
  const double snu = std::sqrt(static_cast<double>(nu));
  for (int i = 0; i < m * m; ++i) {
    Lnu[i] = static_cast<float>(snu * L[i]);
    R_out[i] = static_cast<float>(Rd[i]);
  }
  return nullptr;
}

}  // namespace host
}  // namespace mppi
