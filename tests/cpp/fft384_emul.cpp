// CPU emulation of the 384-point transform of fft.cuh (radix-3 stage, then the 128-point
// radix-16 and radix-8 passes of each row), thread by thread in barrier order, against
// a direct DFT in double precision.  Prints the relative error for several inputs.
#include <array>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "../../paper_2408_03204_b300/csrc/fft.cuh"

using namespace grafx;

int main() {
  constexpr int N = 384;
  std::vector<float2_> cs(N), tw(7 * 16);
  for (int m = 0; m < N; ++m) {
    const double a = 2.0 * M_PI * m / N;
    cs[m] = float2_{float(std::cos(a)), float(std::sin(a))};
  }
  for (int r = 1; r < 8; ++r)
    for (int k = 0; k < 16; ++k) {
      const double a = -2.0 * M_PI * double(r * k) / 128.0;
      tw[(r - 1) * 16 + k] = float2_{float(std::cos(a)), float(std::sin(a))};
    }
  std::mt19937 g(7);
  std::normal_distribution<double> nd;
  double worst = 0;
  for (int trial = 0; trial < 4; ++trial) {
    std::vector<double> xr(N), xi(N);
    std::vector<float2> buf(3 * fft::R128);
    for (int j = 0; j < N; ++j) {
      // trial 0: a single impulse; 1: one complex exponential; else noise
      xr[j] = trial == 0 ? (j == 5) : trial == 1 ? std::cos(2 * M_PI * 37 * j / N) : float(nd(g));
      xi[j] = trial == 0 ? 0.0 : trial == 1 ? std::sin(2 * M_PI * 37 * j / N) : float(nd(g));
      xr[j] = float(xr[j]);
      xi[j] = float(xi[j]);
      buf[fft::in384(j)] = make_float2(float(xr[j]), float(xi[j]));
    }
    for (int j2 = 0; j2 < 128; ++j2) fft::r3_stage384(buf.data(), j2, cs.data());
    for (int row = 0; row < 3; ++row) {
      float2* rb = buf.data() + row * fft::R128;
      std::array<std::array<float2, 16>, 8> v16;
      for (int t = 0; t < 8; ++t) fft::pass_load<128, 16>(rb, t, reinterpret_cast<float2(*)[16]>(v16[t].data()));
      for (int t = 0; t < 8; ++t) fft::pass_store<128, 16>(rb, tw.data(), t, 1, reinterpret_cast<float2(*)[16]>(v16[t].data()));
      std::array<std::array<float2, 16>, 8> v8;
      for (int t = 0; t < 8; ++t) fft::pass_load<128, 8>(rb, t, reinterpret_cast<float2(*)[8]>(v8[t].data()));
      for (int t = 0; t < 8; ++t) fft::pass_store<128, 8>(rb, tw.data(), t, 16, reinterpret_cast<float2(*)[8]>(v8[t].data()));
    }
    double err = 0, ref = 0;
    for (int k = 0; k < N; ++k) {
      double sr = 0, si = 0;
      for (int n = 0; n < N; ++n) {
        const double a = -2.0 * M_PI * double((k * n) % N) / N;
        sr += xr[n] * std::cos(a) - xi[n] * std::sin(a);
        si += xr[n] * std::sin(a) + xi[n] * std::cos(a);
      }
      const float2 y = buf[fft::out384(k)];
      err = std::max(err, std::hypot(y.x - sr, y.y - si));
      ref = std::max(ref, std::hypot(sr, si));
    }
    std::printf("%d %.3e\n", trial, err / ref);
    worst = std::max(worst, err / ref);
  }
  return worst < 1e-6 ? 0 : 1;
}
