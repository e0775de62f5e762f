// Host check of the FP32-seeded FP64 refinements used by the mixed-precision
// inversion (sqrt_from_f32, rcp_from_f32: one Newton step from an FP32 seed)
// against the C library's correctly rounded sqrt and division. Prints the
// largest relative errors over log-uniform samples of the ranges the
// inversion uses.
#include <cmath>
#include <cstdio>
#include <random>

#include "kh_physics.cuh"

int main() {
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  double es = 0.0, er = 0.0;
  for (int n = 0; n < 2000000; ++n) {
    const double x = std::exp(std::log(1e-16) * u(rng));   // 1 - v^2 in [1e-16, 1]
    const double y = std::exp(std::log(1e-30) + std::log(1e60) * u(rng));  // FP32 normal range
    const double s = kh::sqrt_from_f32(x), r = kh::rcp_from_f32(y);
    es = std::fmax(es, std::fabs(s - std::sqrt(x)) / std::sqrt(x));
    er = std::fmax(er, std::fabs(r - 1.0 / y) * y);
  }
  std::printf("%.3e %.3e\n", es, er);
  return 0;
}
