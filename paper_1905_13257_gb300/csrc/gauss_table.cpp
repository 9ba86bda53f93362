// Quantile table of the counter-based Gaussian (host side).
//
// The paper draws Psi and Omega with i.i.d. Gaussian entries (Sec. 2.2,
// Algorithm 4 step 3) without naming a generator.  This library maps a 12-bit
// uniform field u to q[u] = bf16_rn(Phi^{-1}((u + 0.5) / 4096)): the mid-point
// quantile of the standard normal, rounded to nearest-even bfloat16 directly
// from FP64.  Device code then needs no transcendental function and every
// entry is exact in bfloat16, FP32 and FP64.
//
// Phi^{-1} is Wichura's algorithm AS 241 (PPND16), Applied Statistics 37(3),
// 1988: a rational approximation in three ranges with relative accuracy about
// 1e-16, far below the bfloat16 rounding step.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "idsk_internal.h"

namespace {

double poly8(const double* c, double r) {
  double v = c[7];
  for (int i = 6; i >= 0; --i) v = v * r + c[i];
  return v;
}

// AS 241 coefficients: numerators a, c, e and denominators b, d, f
// (denominators have constant term 1).
const double kA[8] = {3.3871328727963666080e0, 1.3314166789178437745e+2,
                      1.9715909503065514427e+3, 1.3731693765509461125e+4,
                      4.5921953931549871457e+4, 6.7265770927008700853e+4,
                      3.3430575583588128105e+4, 2.5090809287301226727e+3};
const double kB[8] = {1.0, 4.2313330701600911252e+1, 6.8718700749205790830e+2,
                      5.3941960214247511077e+3, 2.1213794301586595867e+4,
                      3.9307895800092710610e+4, 2.8729085735721942674e+4,
                      5.2264952788528545610e+3};
const double kC[8] = {1.42343711074968357734e0, 4.63033784615654529590e0,
                      5.76949722146069140550e0, 3.64784832476320460504e0,
                      1.27045825245236838258e0, 2.41780725177450611770e-1,
                      2.27238449892691845833e-2, 7.74545014278341407640e-4};
const double kD[8] = {1.0, 2.05319162663775882187e0, 1.67638483018380384940e0,
                      6.89767334985100004550e-1, 1.48103976427480074590e-1,
                      1.51986665636164571966e-2, 5.47593808499534494600e-4,
                      1.05075007164441684324e-9};
const double kE[8] = {6.65790464350110377720e0, 5.46378491116411436990e0,
                      1.78482653991729133580e0, 2.96560571828504891230e-1,
                      2.65321895265761230930e-2, 1.24266094738807843860e-3,
                      2.71155556874348757815e-5, 2.01033439929228813265e-7};
const double kF[8] = {1.0, 5.99832206555887937690e-1, 1.36929880922735805310e-1,
                      1.48753612908506148525e-2, 7.86869131145613259100e-4,
                      1.84631831751005468180e-5, 1.42151175831644588870e-7,
                      2.04426310338993978564e-15};

double ppnd16(double p) {
  const double q = p - 0.5;
  if (fabs(q) <= 0.425) {
    const double r = 0.180625 - q * q;
    return q * poly8(kA, r) / poly8(kB, r);
  }
  double r = q < 0.0 ? p : 1.0 - p;
  r = sqrt(-log(r));
  double v;
  if (r <= 5.0) {
    r -= 1.6;
    v = poly8(kC, r) / poly8(kD, r);
  } else {
    r -= 5.0;
    v = poly8(kE, r) / poly8(kF, r);
  }
  return q < 0.0 ? -v : v;
}

// Nearest-even rounding of a finite normal double to 8 significant bits.
double round_to_bf16(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  const uint64_t low = (uint64_t(1) << 45) - 1;        // mantissa bits dropped
  const uint64_t keep_lsb = (b >> 45) & 1u;
  b = (b + (low >> 1) + keep_lsb) & ~low;
  double r;
  memcpy(&r, &b, 8);
  return r;
}

}  // namespace

namespace idsk {

void gaussian_table_host(float* vals, uint16_t* bits) {
  for (int u = 0; u < kTableSize; ++u) {
    const double q = round_to_bf16(ppnd16((u + 0.5) / kTableSize));
    const float f = (float)q;   // exact
    uint32_t fb;
    memcpy(&fb, &f, 4);
    if (vals) vals[u] = f;
    if (bits) bits[u] = (uint16_t)(fb >> 16);
  }
}

}  // namespace idsk
