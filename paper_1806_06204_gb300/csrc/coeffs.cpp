// Zolotarev coefficients and the a-priori iteration schedule (host, FP64).
//
// Eq. (7):  c_i = l^2 sn^2(u_i; l') / cn^2(u_i; l'),  u_i = i K' / (2r+1),
//           l' = sqrt(1 - l^2),  K' = K(l') the complete elliptic integral.
// Eq. (8):  Zhat(x) = M_hat x prod_j (x^2 + c_{2j}) / (x^2 + c_{2j-1}),
//           M_hat = prod_j (1 + c_{2j-1}) / (1 + c_{2j}).
// Eq. (10): a_j, the residue of Zhat / (M_hat x) at x^2 = -c_{2j-1}:
//           a_j = -prod_k (c_{2j-1} - c_{2k}) / prod_{k != j} (c_{2j-1} - c_{2k-1})
//           (the paper prints a product of the two products; the partial
//           fraction expansion of Eq. (9) needs their quotient).
// Algorithm 1 step (c): l <- Zhat(l; l) (printed with l + c_{2j} in the
//           numerator; Eq. (8) at x = l has l^2 + c_{2j}).
// Table 1:  iterate until 1 - l <= 1e-15.
//
// Evaluation: the ratio sc = sn/cn at modulus l' equals -i sn(iu; l) (Jacobi's
// imaginary transformation, Abramowitz & Stegun 16.20.1).  sn at the small
// modulus l is evaluated by the descending Landen / AGM scale (A&S 16.4); with
// an imaginary phase the backward phase recurrence is real in asinh/sinh form.
// Arguments beyond K'/2 use the quarter-period reflection
// sc(K' - v; l') = 1 / (l sc(v; l')) (A&S 16.8).  K' = pi / (2 AGM(1, l))
// (A&S 17.6).  No step subtracts nearly equal numbers, so l down to 1e-300
// is handled.
//
// 1 - Zhat(l; l) is evaluated in factored form: on [l, 1], 1 - Zhat(x) >= 0
// vanishes at x = 1 and doubly at the r interior maxima x_m with
// x_m^2 = (l^2 + c_{2m-1}) / (1 + c_{2m-1}) (the points l / dn(u_{2m-1}; l')),
// so 1 - Zhat(l) = M_hat (1 - l) prod_m (x_m - l)^2 / prod_m (l^2 + c_{2m-1}).
#include <cmath>
#include <cstddef>

#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr double kPi = 3.14159265358979323846;

struct AgmScale {
  int steps = 0;
  double a[64];
  double c[64];
};

// AGM scale for the modulus k = l with complementary modulus k' = l':
// a_0 = 1, b_0 = l', c_0 = l; c_{n} = c_{n-1}^2 / (4 a_n) avoids (a - b)/2.
AgmScale agm_scale(double ell) {
  AgmScale s;
  double a = 1.0, b = std::sqrt((1.0 - ell) * (1.0 + ell)), c = ell;
  s.a[0] = a;
  s.c[0] = c;
  while (c > kEps * a && s.steps < 62) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    c = c * c / (4.0 * an);
    a = an;
    ++s.steps;
    s.a[s.steps] = a;
    s.c[s.steps] = c;
  }
  return s;
}

// asinh(x sinh(psi)), x > 0, psi >= 0, safe for large psi.
double asinh_scaled_sinh(double x, double psi) {
  if (psi < 30.0) return std::asinh(x * std::sinh(psi));
  const double log_y = std::log(x) + psi - std::log(2.0) + std::log1p(-std::exp(-2.0 * psi));
  const double inv_y2 = log_y < 300.0 ? std::exp(-2.0 * log_y) : 0.0;
  return std::log(2.0) + log_y + std::log(0.5 * (1.0 + std::sqrt(1.0 + inv_y2)));
}

// sc(u; l') for 0 <= u <= K'/2 from the precomputed AGM scale of modulus l.
double sc_half_period(const AgmScale& s, double u) {
  double psi = std::ldexp(s.a[s.steps] * u, s.steps);
  for (int n = s.steps; n >= 1; --n) psi = 0.5 * (psi + asinh_scaled_sinh(s.c[n] / s.a[n], psi));
  return std::sinh(psi);
}

double agm_mean(double a, double b) {
  for (int it = 0; it < 200 && std::fabs(a - b) > 2.0 * kEps * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return 0.5 * (a + b);
}

}  // namespace

int compute_coefficients(double ell, int r, Coefficients* out) {
  if (!(ell > 0.0 && ell <= 1.0)) return -1;
  if (r < 1 || r > kMaxR) return -2;
  out->ell = ell;
  out->r = r;
  const int two_r1 = 2 * r + 1;
  double* c = out->c;
  if (ell == 1.0) {
    // modulus l' = 0: sc = tan, K' = pi/2 (the limit of Eq. (7))
    for (int i = 1; i <= 2 * r; ++i) {
      const double t = std::tan(i * (kPi / 2.0) / two_r1);
      c[i - 1] = t * t;
    }
  } else {
    const AgmScale s = agm_scale(ell);
    const double Kp = kPi / (2.0 * agm_mean(1.0, ell));
    for (int i = 1; i <= 2 * r; ++i) {
      if (2 * i <= two_r1) {
        const double v = sc_half_period(s, i * Kp / two_r1);
        c[i - 1] = ell * ell * v * v;
      } else {
        const double v = sc_half_period(s, (two_r1 - i) * Kp / two_r1);
        c[i - 1] = 1.0 / (v * v);
      }
    }
  }
  double mhat = 1.0;
  for (int j = 0; j < r; ++j) mhat *= (1.0 + c[2 * j]) / (1.0 + c[2 * j + 1]);
  out->mhat = mhat;
  for (int j = 0; j < r; ++j) {
    const double codd = c[2 * j];
    double num = 1.0, den = 1.0;
    for (int k = 0; k < r; ++k) {
      num *= codd - c[2 * k + 1];
      if (k != j) den *= codd - c[2 * k];
    }
    out->a[j] = -num / den;
  }
  // 1 - Zhat(l; l) in factored form (see the file comment)
  const double lp2 = (1.0 - ell) * (1.0 + ell);
  double gap = mhat * (1.0 - ell);
  for (int m = 0; m < r; ++m) {
    const double codd = c[2 * m];
    const double xm = std::sqrt((ell * ell + codd) / (1.0 + codd));
    const double d = codd * lp2 / ((1.0 + codd) * (xm + ell));
    gap *= d * d / (ell * ell + codd);
  }
  out->gap = gap;
  return 0;
}

bool qr_form_needed(const Coefficients& co) {
  // kappa(Z_1) <= (1 + c_1) / (l^2 + c_1): use the Cholesky form once it is <= 100
  return (1.0 + co.c[0]) / (co.ell * co.ell + co.c[0]) > 100.0;
}

int build_schedule(double ell0, int r, int max_iter, Schedule* out) {
  if (!(ell0 > 0.0 && ell0 <= 1.0)) return -1;
  if (r < 0 || r > kMaxR) return -2;
  if (max_iter < 1 || max_iter > kMaxIters) return -3;
  if (r == 0) {
    // smallest r <= 8 whose schedule has at most two iterations (Table 1 guidance)
    for (r = 1; r < kMaxR; ++r) {
      Schedule probe;
      build_schedule(ell0, r, kMaxIters, &probe);
      if (probe.iters <= 2) break;
    }
  }
  out->r = r;
  out->ell[0] = ell0;
  double gap = 1.0 - ell0;
  int k = 0;
  while (gap > kTable1Tol && k < max_iter) {
    Coefficients co;
    compute_coefficients(out->ell[k], r, &co);
    out->co[k] = co;
    out->use_qr[k] = qr_form_needed(co);
    gap = co.gap;
    out->ell[k + 1] = 1.0 - gap;
    ++k;
  }
  out->iters = k;
  out->converged = gap <= kTable1Tol;
  return 0;
}

}  // namespace zolo
