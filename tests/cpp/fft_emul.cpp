// CPU emulation of the shared-memory FFT passes (fft.cuh): runs every thread's load
// phase, then every thread's store phase, exactly as the barriers order them on the
// GPU, and compares the result with a direct O(M^2) DFT in double precision.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "../../paper_2408_03204_b300/csrc/fft.cuh"

using namespace grafx;

template <int M, int R>
void run_pass(std::vector<float2>& buf, const std::vector<float2_>& tw, int Ns, int pass) {
  constexpr int T = M / 16;
  const float2_* twp = tw.data() + fft::ptw_base(M) + fft::ptw_pass_off(M, pass);
  std::vector<std::array<std::array<float2, R>, 16 / R>> v(T);
  for (int t = 0; t < T; ++t) fft::pass_load<M, R>(buf.data(), t, reinterpret_cast<float2(*)[R]>(v[t].data()));
  for (int t = 0; t < T; ++t) fft::pass_store<M, R>(buf.data(), twp, t, Ns, reinterpret_cast<float2(*)[R]>(v[t].data()));
}

template <int M>
double check(std::mt19937& g, const std::vector<float2_>& tw) {
  std::normal_distribution<double> nd;
  std::vector<double> xr(M), xi(M);
  std::vector<float2> buf(fft::Padded<M>::size);
  for (int i = 0; i < M; ++i) {
    xr[i] = float(nd(g)); xi[i] = float(nd(g));
    buf[fft::pad(i)] = make_float2(float(xr[i]), float(xi[i]));
  }
  int Ns = 1;
  for (int p = 0; p < fft::Geo<M>::n16; ++p) { run_pass<M, 16>(buf, tw, Ns, p); Ns *= 16; }
  if constexpr (fft::Geo<M>::last > 1) run_pass<M, fft::Geo<M>::last>(buf, tw, Ns, fft::Geo<M>::n16);
  double err = 0, ref = 0;
  for (int k = 0; k < M; ++k) {
    double sr = 0, si = 0;
    for (int n = 0; n < M; ++n) {
      double a = -2.0 * M_PI * double((int64_t(k) * n) % M) / M;
      sr += xr[n] * std::cos(a) - xi[n] * std::sin(a);
      si += xr[n] * std::sin(a) + xi[n] * std::cos(a);
    }
    float2 y = buf[fft::pad(k)];
    err = std::max(err, std::hypot(y.x - sr, y.y - si));
    ref = std::max(ref, std::hypot(sr, si));
  }
  return err / ref;
}

int main() {
  // pass twiddle tables: W_{Ns R}^{r k} at [(r-1) Ns + k], concatenated over M
  std::vector<float2_> tw(fft::PTW_TOTAL);
  for (int M = 512; M <= 8192; M *= 2)
    for (int pass = 1, Ns = 16; pass < fft::geo_npass(M); ++pass, Ns *= 16) {
      const int R = fft::pass_radix(M, pass);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          double a = -2.0 * M_PI * double(r) * k / (double(Ns) * R);
          tw[fft::ptw_base(M) + fft::ptw_pass_off(M, pass) + (r - 1) * Ns + k] = float2_{float(std::cos(a)), float(std::sin(a))};
        }
    }
  std::mt19937 g(5);
  std::printf("512 %.3e\n", check<512>(g, tw));
  std::printf("1024 %.3e\n", check<1024>(g, tw));
  std::printf("2048 %.3e\n", check<2048>(g, tw));
  std::printf("4096 %.3e\n", check<4096>(g, tw));
  std::printf("8192 %.3e\n", check<8192>(g, tw));
  return 0;
}
