// A kernel basis of a general A, host side: Lemma 3.1 (unimodular column
// operations K with A K = (H | 0); the last d = n - m columns of K span
// Ker_Z(A), Theorem 3.2), optionally reduced by LLL (Appendix A).
//
// HNF: row by row, the entries right of the pivot are cleared by
// extended-gcd combinations of two columns (128-bit integers; an entry
// beyond 2^62 is reported as SHAPE), a negative pivot column is negated.
// LLL: columns are size-reduced against their predecessors (mu rounded to
// the nearest integer, halves away from zero) and adjacent columns exchanged
// while ||B*_{i-1}||^2 > 2 ||B*_i||^2 (the appendix's condition (ii)).  The
// Gram-Schmidt data are IEEE double (so x86 and Arm hosts agree); a
// column's row is recomputed from the integer vectors before it is reduced,
// and the reduction repeats until no coefficient rounds away from zero, so
// that large entries of the unreduced basis do not leave stale coefficients.
#include "common.cuh"

#include <cmath>
#include <vector>

namespace {

typedef __int128 i128;
constexpr i128 kLimit = (i128)1 << 62;

void egcd(i128 a, i128 b, i128& g, i128& x, i128& y) {
  i128 x0 = 1, y0 = 0, x1 = 0, y1 = 1;
  while (b != 0) {
    // floor division, as Python's //
    i128 q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    const i128 r = a - q * b;
    a = b;
    b = r;
    const i128 tx = x0 - q * x1, ty = y0 - q * y1;
    x0 = x1; x1 = tx;
    y0 = y1; y1 = ty;
  }
  if (a < 0) { a = -a; x0 = -x0; y0 = -y0; }
  g = a; x = x0; y = y0;
}

i128 floordiv(i128 a, i128 b) {
  i128 q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

}  // namespace

extern "C" int mape_kernel_basis(int32_t m, int32_t n, const int32_t* A, int32_t reduce, int32_t* B_out) {
  if (m <= 0 || n <= m || !A || !B_out) return MAPE_ERR_INVALID_ARG;
  const int d = n - m;
  std::vector<i128> M((size_t)m * n), K((size_t)n * n, 0);
  for (size_t e = 0; e < M.size(); ++e) M[e] = A[e];
  for (int i = 0; i < n; ++i) K[(size_t)i * n + i] = 1;
  // col_c <- x col_c + y col_j, col_j <- p col_c + q col_j, in M and K
  auto combine = [&](int c, int j, i128 x, i128 y, i128 p, i128 q) -> bool {
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<i128>& R = pass ? K : M;
      const int rows = pass ? n : m;
      for (int r = 0; r < rows; ++r) {
        const i128 a = R[(size_t)r * n + c], b = R[(size_t)r * n + j];
        const i128 na = x * a + y * b, nb = p * a + q * b;
        if (na > kLimit || na < -kLimit || nb > kLimit || nb < -kLimit) return false;
        R[(size_t)r * n + c] = na;
        R[(size_t)r * n + j] = nb;
      }
    }
    return true;
  };
  for (int i = 0; i < m; ++i) {
    const int c = i;
    for (int j = c + 1; j < n; ++j) {
      const i128 b = M[(size_t)i * n + j];
      if (b == 0) continue;
      const i128 a = M[(size_t)i * n + c];
      i128 g, x, y;
      egcd(a, b, g, x, y);
      if (!combine(c, j, x, y, floordiv(-b, g), floordiv(a, g))) return MAPE_ERR_SHAPE;
    }
    if (M[(size_t)i * n + c] == 0) return MAPE_ERR_INVALID_ARG;  // A is not of full row rank
    if (M[(size_t)i * n + c] < 0) {
      for (int r = 0; r < m; ++r) M[(size_t)r * n + c] = -M[(size_t)r * n + c];
      for (int r = 0; r < n; ++r) K[(size_t)r * n + c] = -K[(size_t)r * n + c];
    }
  }
  // basis columns: K's last d columns, as int64 column vectors
  std::vector<std::vector<long long>> b(d, std::vector<long long>(n));
  for (int j = 0; j < d; ++j)
    for (int r = 0; r < n; ++r) b[j][r] = (long long)K[(size_t)r * n + m + j];
  if (reduce) {
    std::vector<std::vector<double>> mu(d, std::vector<double>(d, 0.0));
    std::vector<double> Bn(d, 0.0);
    std::vector<std::vector<double>> star(d, std::vector<double>(n));
    // Gram-Schmidt row i from the current integer column b_i and the stored
    // rows j < i (never from stale incremental updates)
    auto compute_row = [&](int i) {
      for (int r = 0; r < n; ++r) star[i][r] = (double)b[i][r];
      for (int j = 0; j < i; ++j) {
        double s2 = 0.0;
        for (int r = 0; r < n; ++r) s2 += (double)b[i][r] * star[j][r];
        mu[i][j] = Bn[j] > 0.0 ? s2 / Bn[j] : 0.0;
        for (int r = 0; r < n; ++r) star[i][r] -= mu[i][j] * star[j][r];
      }
      double s2 = 0.0;
      for (int r = 0; r < n; ++r) s2 += star[i][r] * star[i][r];
      Bn[i] = s2;
    };
    // nearest integer, halves away from zero; a coefficient within 1e-9 of a
    // half-integer is such a half in exact arithmetic (small integer data)
    auto nearest = [](double q) {
      const double a = std::fabs(q) + 1e-9;
      const double k = std::floor(a + 0.5);
      return q >= 0 ? k : -k;
    };
    // size reduction of column i, repeated until no coefficient rounds away
    // from zero (large quotients leave rounding residue in one pass)
    auto size_reduce = [&](int i) -> bool {
      for (int pass = 0; pass < 64; ++pass) {
        compute_row(i);
        bool changed = false;
        for (int j = i - 1; j >= 0; --j) {
          // the first pass is the reduction itself; later passes only remove
          // floating-point residue (a coefficient of exactly one half stays)
          if (pass > 0 && std::fabs(mu[i][j]) <= 0.5 + 1e-6) continue;
          const double q = nearest(mu[i][j]);
          if (q == 0.0) continue;
          if (std::fabs(q) > 4.0e18) return false;
          const long long qi = (long long)q;
          for (int r = 0; r < n; ++r) {
            const i128 v = (i128)b[i][r] - (i128)qi * b[j][r];
            if (v > kLimit || v < -kLimit) return false;
            b[i][r] = (long long)v;
          }
          for (int k = 0; k < j; ++k) mu[i][k] -= q * mu[j][k];
          mu[i][j] -= q;
          changed = true;
        }
        if (!changed) return true;
      }
      return true;
    };
    compute_row(0);
    int i = 1;
    long long guard = 0;
    while (i < d) {
      if (++guard > 100000000LL) return MAPE_ERR_NUMERIC;
      if (!size_reduce(i)) return MAPE_ERR_SHAPE;
      if (Bn[i - 1] > 2.0 * Bn[i]) {
        std::swap(b[i - 1], b[i]);
        compute_row(i - 1);  // rows below i - 1 are unchanged; row i is recomputed when reached
        i = i - 1 > 1 ? i - 1 : 1;
        if (i == 1) compute_row(0);
      } else {
        ++i;
      }
    }
  }
  for (int j = 0; j < d; ++j)
    for (int r = 0; r < n; ++r) {
      if (b[j][r] > INT32_MAX || b[j][r] < INT32_MIN) return MAPE_ERR_SHAPE;
      B_out[(size_t)r * d + j] = (int32_t)b[j][r];
    }
  // exact check A B = 0
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < d; ++j) {
      long long s = 0;
      for (int k = 0; k < n; ++k) s += (long long)A[(size_t)r * n + k] * B_out[(size_t)k * d + j];
      if (s != 0) return MAPE_ERR_NUMERIC;
    }
  return MAPE_OK;
}
