// Linear inequalities G x >= h (§3.4, Corollary 3.3), host side: the
// equality form with slack s = G x - h >= 0, constraint matrix [A 0; G -I],
// right-hand side (b, h) and kernel basis [B; G B].  x is boxed, so each
// slack is bounded above by its largest value over the box,
// max_x (G x)_k - h_k; the extended instance then runs on every stage as it
// is (its basis keeps B's identity top).
#include "common.cuh"

#include <cstring>

extern "C" int mape_inequality_extension(int32_t n, int32_t m, int32_t m2, const int32_t* A, const int64_t* b,
                                         const int32_t* l, const int32_t* u, const int32_t* G, const int64_t* h,
                                         const int32_t* B, int32_t* A2, int64_t* b2, int32_t* l2, int32_t* u2,
                                         int32_t* B2) {
  if (n <= 0 || m < 0 || m >= n || m2 <= 0 || !A || !b || !l || !u || !G || !h || !B || !A2 || !b2 || !l2 || !u2 ||
      !B2)
    return MAPE_ERR_INVALID_ARG;
  const int d = n - m, n2 = n + m2, mm = m + m2;
  // G B must stay in int32
  for (int k = 0; k < m2; ++k)
    for (int j = 0; j < d; ++j) {
      long long acc = 0;
      for (int i = 0; i < n; ++i) acc += (long long)G[(int64_t)k * n + i] * B[(int64_t)i * d + j];
      if (acc > INT32_MAX || acc < INT32_MIN) return MAPE_ERR_SHAPE;
      B2[(int64_t)(n + k) * d + j] = (int32_t)acc;
    }
  std::memcpy(B2, B, sizeof(int32_t) * (size_t)n * d);
  for (int k = 0; k < m2; ++k) {
    long long smax = -h[k];
    for (int i = 0; i < n; ++i) {
      const long long g = G[(int64_t)k * n + i];
      smax += g * (g > 0 ? u[i] : l[i]);
    }
    if (smax < 0) return MAPE_ERR_BOUNDS;  // no point of the box satisfies inequality k
    if (smax > INT32_MAX) return MAPE_ERR_SHAPE;
    l2[n + k] = 0;
    u2[n + k] = (int32_t)smax;
  }
  std::memcpy(l2, l, sizeof(int32_t) * n);
  std::memcpy(u2, u, sizeof(int32_t) * n);
  std::memset(A2, 0, sizeof(int32_t) * (size_t)mm * n2);
  for (int r = 0; r < m; ++r) std::memcpy(A2 + (int64_t)r * n2, A + (int64_t)r * n, sizeof(int32_t) * n);
  for (int k = 0; k < m2; ++k) {
    std::memcpy(A2 + (int64_t)(m + k) * n2, G + (int64_t)k * n, sizeof(int32_t) * n);
    A2[(int64_t)(m + k) * n2 + n + k] = -1;
  }
  std::memcpy(b2, b, sizeof(int64_t) * m);
  std::memcpy(b2 + m, h, sizeof(int64_t) * m2);
  return MAPE_OK;
}

// The objective of the extended instance: f of the first n coordinates, the
// slacks enter neither Q, c nor w.
extern "C" int mape_inequality_extension_objective(int32_t n, int32_t m2, const int32_t* Q, const int32_t* c,
                                                   const int32_t* w, int32_t* Q2, int32_t* c2, int32_t* w2) {
  if (n <= 0 || m2 <= 0 || !Q || !c || !Q2 || !c2 || (w && !w2)) return MAPE_ERR_INVALID_ARG;
  const int n2 = n + m2;
  std::memset(Q2, 0, sizeof(int32_t) * (size_t)n2 * n2);
  for (int i = 0; i < n; ++i) std::memcpy(Q2 + (int64_t)i * n2, Q + (int64_t)i * n, sizeof(int32_t) * n);
  std::memcpy(c2, c, sizeof(int32_t) * n);
  std::memset(c2 + n, 0, sizeof(int32_t) * m2);
  if (w) {
    std::memcpy(w2, w, sizeof(int32_t) * n);
    std::memset(w2 + n, 0, sizeof(int32_t) * m2);
  }
  return MAPE_OK;
}

// Points of the extended instance: x followed by its slacks s = G x - h.
extern "C" int mape_inequality_extension_points(int32_t n, int32_t m2, const int32_t* G, const int64_t* h,
                                                const int32_t* X, int32_t S, int32_t* X2) {
  if (n <= 0 || m2 <= 0 || S < 0 || !G || !h || (S > 0 && (!X || !X2))) return MAPE_ERR_INVALID_ARG;
  const int n2 = n + m2;
  for (int s = 0; s < S; ++s) {
    const int32_t* x = X + (int64_t)s * n;
    int32_t* y = X2 + (int64_t)s * n2;
    std::memcpy(y, x, sizeof(int32_t) * n);
    for (int k = 0; k < m2; ++k) {
      long long v = -h[k];
      for (int i = 0; i < n; ++i) v += (long long)G[(int64_t)k * n + i] * x[i];
      if (v < 0) return MAPE_ERR_BOUNDS;  // x violates inequality k: no slack exists
      if (v > INT32_MAX) return MAPE_ERR_SHAPE;
      y[n + k] = (int32_t)v;
    }
  }
  return MAPE_OK;
}
