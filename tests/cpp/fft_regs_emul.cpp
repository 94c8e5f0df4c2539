// CPU emulation of fft::forward_regs (fft.cuh): the register-resident first and last
// passes with ping-pong shared buffers, run thread by thread in barrier order, against
// a direct DFT in double precision.  Checks the register layout x[tid + T m] on entry
// and X[tid + T m] on exit.
#include <array>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "../../paper_2408_03204_b300/csrc/fft.cuh"

using namespace grafx;

template <int M>
double check(std::mt19937& g, const std::vector<float2_>& tw) {
  constexpr int T = M / 16, n16 = fft::Geo<M>::n16, last = fft::Geo<M>::last;
  constexpr int npass = n16 + (last > 1 ? 1 : 0);
  std::normal_distribution<double> nd;
  std::vector<double> xr(M), xi(M);
  std::vector<std::array<float2, 16>> v(T);
  for (int i = 0; i < M; ++i) { xr[i] = float(nd(g)); xi[i] = float(nd(g)); }
  for (int t = 0; t < T; ++t)
    for (int m = 0; m < 16; ++m) v[t][m] = make_float2(float(xr[t + T * m]), float(xi[t + T * m]));
  std::vector<float2> b[2] = {std::vector<float2>(fft::Padded<M>::size), std::vector<float2>(fft::Padded<M>::size)};
  for (int t = 0; t < T; ++t) {
    fft::Dft<16>::run(v[t].data());
    for (int r = 0; r < 16; ++r) b[0][fft::pad(t * 16 + r)] = v[t][r];
  }
  int Ns = 16, cur = 0;
  for (int p = 1; p < npass; ++p) {
    const bool is_last = p == npass - 1;
    const int R = (is_last && last > 1) ? last : 16;
    if (R == 16) {
      std::vector<std::array<float2, 16>> w(T);
      for (int t = 0; t < T; ++t) fft::pass_load<M, 16>(b[cur].data(), t, reinterpret_cast<float2(*)[16]>(w[t].data()));
      for (int t = 0; t < T; ++t) {
        fft::pass_compute<M, 16>(tw.data() + fft::ptw_base(M) + fft::ptw_pass_off(M, p), t, Ns, reinterpret_cast<float2(*)[16]>(w[t].data()));
        if (is_last) { v[t] = w[t]; continue; }
        int k = t & (Ns - 1), out = (t - k) * 16 + k;
        for (int r = 0; r < 16; ++r) b[cur ^ 1][fft::pad(out + r * Ns)] = w[t][r];
      }
    } else if constexpr (last > 1 && last < 16) {
      constexpr int RL = last, BPT = 16 / RL;
      std::vector<std::array<float2, 16>> w(T);
      for (int t = 0; t < T; ++t) {
        auto* ww = reinterpret_cast<float2(*)[RL]>(w[t].data());
        fft::pass_load<M, RL>(b[cur].data(), t, ww);
        fft::pass_compute<M, RL>(tw.data() + fft::ptw_base(M) + fft::ptw_pass_off(M, p), t, Ns, ww);
        for (int bb = 0; bb < BPT; ++bb)
          for (int r = 0; r < RL; ++r) v[t][bb + r * BPT] = ww[bb][r];
      }
    }
    if (!is_last) { cur ^= 1; Ns *= 16; }
  }
  double err = 0, ref = 0;
  for (int k = 0; k < M; ++k) {
    double sr = 0, si = 0;
    for (int n = 0; n < M; ++n) {
      double a = -2.0 * M_PI * double((int64_t(k) * n) % M) / M;
      sr += xr[n] * std::cos(a) - xi[n] * std::sin(a);
      si += xr[n] * std::sin(a) + xi[n] * std::cos(a);
    }
    float2 y = v[k % T][k / T];
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
  std::mt19937 g(7);
  std::printf("512 %.3e\n", check<512>(g, tw));
  std::printf("1024 %.3e\n", check<1024>(g, tw));
  std::printf("2048 %.3e\n", check<2048>(g, tw));
  std::printf("4096 %.3e\n", check<4096>(g, tw));
  std::printf("8192 %.3e\n", check<8192>(g, tw));
  return 0;
}
