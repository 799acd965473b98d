// Host program for tests/test_fft_core.py: runs the row-FFT building blocks of
// csrc/fft_core.h on the CPU, with the same pass schedule as the device kernels
// (one pass of radix 2^(L mod 4) first when L is not a multiple of 4, then radix-16
// passes), emulating the block barrier between the load and store halves of a pass.
//
// stdin:  mode L count, then the input numbers (mode c2c/ic2c: 2*2^L reals as
//         interleaved complex; r2c: 2^(L+1) reals; c2r: 2*(2^L + 1) reals, the half
//         spectrum X[0..N2]).  fc2c/fic2c: c2c/ic2c in float (the FP32 plans' arithmetic);
//         dc2c/dic2c: in float-float (the GP_DF64 plans' arithmetic, ff64.h).
// stdout: the output numbers, one per line (c2c/ic2c: 2*2^L; r2c: 2*(2^L + 1);
//         c2r: 2^(L+1) reals).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fft_core.h"

using gpn::fft::cpx;
using gpn::fft::Pass;
using C = cpx<double>;

// a pass with the two-level twiddle (the real split's functor), for the radix-2/4/8 pass
template <int R, int NB, bool INV, typename T = double>
void pass2(std::vector<cpx<T>>& buf, int N, int Ns) {
  const int nt = N / 16;
  std::vector<Pass<R, NB, T>> st(nt);
  for (int t = 0; t < nt; ++t) st[t].load(buf.data(), N, t, nt);
  std::vector<cpx<T>> hi(N / 64 + 1), lo(64);
  for (int q = 0; q < (int)hi.size(); ++q)
    hi[q] = {(T)std::cos(2 * M_PI * (64.0 * q) / N), (T)-std::sin(2 * M_PI * (64.0 * q) / N)};
  for (int j = 0; j < 64; ++j) lo[j] = {(T)std::cos(2 * M_PI * j / N), (T)-std::sin(2 * M_PI * j / N)};
  const gpn::fft::Twiddle2<T> t2{hi.data(), lo.data()};
  for (int t = 0; t < nt; ++t) st[t].template store<INV>(buf.data(), t2, N, Ns, t, nt);
}

// a radix-16 pass with its table from gpn::fft::pass_tables, as on the device
template <bool INV, typename T = double>
void pass16(std::vector<cpx<T>>& buf, const std::vector<cpx<T>>& tab, int L, int Ns) {
  const int N = 1 << L, nt = N / 16;
  std::vector<Pass<16, 1, T>> st(nt);
  for (int t = 0; t < nt; ++t) st[t].load(buf.data(), N, t, nt);
  const gpn::fft::PassTwiddle<T> tw{tab.data() + gpn::fft::pass_table_offset(L, Ns), Ns};
  for (int t = 0; t < nt; ++t) st[t].template store<INV>(buf.data(), tw, N, Ns, t, nt);
}

// the first pass from each thread's registers x[u] = element t + u N/16 (as the device
// row kernels do), then the remaining passes as usual
template <int R, int NB, bool INV>
void first_from_regs(std::vector<C>& buf, int N) {
  const int nt = N / 16;
  std::vector<Pass<R, NB, double>> st(nt);
  for (int t = 0; t < nt; ++t) {
    C x[16];
    for (int u = 0; u < 16; ++u) x[u] = buf[gpn::fft::pad(t + u * nt)];
    gpn::fft::first_pass_inputs(st[t], x);
  }
  const gpn::fft::Twiddle2<double> none{nullptr, nullptr};  // span 1: no twiddles are read
  for (int t = 0; t < nt; ++t) {
    st[t].template compute<INV>(none, N, 1, t, nt);
    st[t].write(buf.data(), 1, t, nt);
  }
}

template <bool INV>
void fft_regs(std::vector<C>& buf, int L) {
  const int N = 1 << L;
  const std::vector<double> raw = gpn::fft::pass_tables(L);
  std::vector<C> tab(raw.size() / 2 + 1);
  for (size_t i = 0; i < raw.size() / 2; ++i) tab[i] = {raw[2 * i], raw[2 * i + 1]};
  int Ns = 1;
  switch (L % 4) {
    case 1: first_from_regs<2, 8, INV>(buf, N); Ns = 2; break;
    case 2: first_from_regs<4, 4, INV>(buf, N); Ns = 4; break;
    case 3: first_from_regs<8, 2, INV>(buf, N); Ns = 8; break;
    default: first_from_regs<16, 1, INV>(buf, N); Ns = 16; break;
  }
  for (int q = (L % 4 == 0) ? 1 : 0; q < L / 4; ++q) {
    pass16<INV>(buf, tab, L, Ns);
    Ns *= 16;
  }
}

template <bool INV, typename T = double>
void fft(std::vector<cpx<T>>& buf, int L) {
  const int N = 1 << L;
  const std::vector<double> raw = gpn::fft::pass_tables(L);
  std::vector<cpx<T>> tab(raw.size() / 2 + 1);
  for (size_t i = 0; i < raw.size() / 2; ++i) tab[i] = {(T)raw[2 * i], (T)raw[2 * i + 1]};
  int Ns = 1;
  switch (L % 4) {
    case 1: pass2<2, 8, INV, T>(buf, N, Ns); Ns *= 2; break;
    case 2: pass2<4, 4, INV, T>(buf, N, Ns); Ns *= 4; break;
    case 3: pass2<8, 2, INV, T>(buf, N, Ns); Ns *= 8; break;
    default: break;
  }
  for (int q = 0; q < L / 4; ++q) {
    pass16<INV, T>(buf, tab, L, Ns);
    Ns *= 16;
  }
}

int main() {
  char mode[16];
  int L;
  if (std::scanf("%15s %d", mode, &L) != 2) return 1;
  const int N = 1 << L;
  std::vector<C> buf(gpn::fft::pad(N) + 1, C{0, 0});
  auto at = [&](int i) -> C& { return buf[gpn::fft::pad(i)]; };
  std::vector<C> wnf(N + 1);
  for (int k = 0; k <= N; ++k) wnf[k] = {std::cos(M_PI * k / N), -std::sin(M_PI * k / N)};  // W_{2N}^k
  if (!std::strcmp(mode, "fc2c") || !std::strcmp(mode, "fic2c")) {
    std::vector<cpx<float>> fb(gpn::fft::pad(N) + 1, cpx<float>{0, 0});
    for (int i = 0; i < N; ++i) {
      double re, im;
      if (std::scanf("%lf %lf", &re, &im) != 2) return 1;
      fb[gpn::fft::pad(i)] = {(float)re, (float)im};
    }
    if (mode[1] == 'i')
      fft<true, float>(fb, L);
    else
      fft<false, float>(fb, L);
    for (int i = 0; i < N; ++i) std::printf("%.9g\n%.9g\n", fb[gpn::fft::pad(i)].x, fb[gpn::fft::pad(i)].y);
    return 0;
  }
  if (!std::strcmp(mode, "dpsi")) {
    // float-float ES kernel (es_psi_dd, as the GP_DF64 kernels evaluate it): "dpsi W"
    // then beta and count, then (j, xi) pairs; prints exp(beta (sqrt(1 - z^2) - 1)),
    // z = (j - xi) 2 / W
    using gpn::dd;
    double beta;
    int n;
    if (std::scanf("%lf %d", &beta, &n) != 2) return 1;
    const dd b(beta), ih(2.0 / L);
    for (int i = 0; i < n; ++i) {
      int j;
      double xi;
      if (std::scanf("%d %lf", &j, &xi) != 2) return 1;
      const dd v = gpn::es_psi_dd(j, dd(xi), b, ih);
      std::printf("%.17g\n", (double)v);
    }
    return 0;
  }
  if (!std::strcmp(mode, "dc2c") || !std::strcmp(mode, "dic2c")) {
    using gpn::dd;
    std::vector<cpx<dd>> fb(gpn::fft::pad(N) + 1, cpx<dd>{dd(0.0), dd(0.0)});
    for (int i = 0; i < N; ++i) {
      double re, im;
      if (std::scanf("%lf %lf", &re, &im) != 2) return 1;
      fb[gpn::fft::pad(i)] = {dd(re), dd(im)};
    }
    if (mode[1] == 'i')
      fft<true, dd>(fb, L);
    else
      fft<false, dd>(fb, L);
    for (int i = 0; i < N; ++i)
      std::printf("%.17g\n%.17g\n", (double)fb[gpn::fft::pad(i)].x, (double)fb[gpn::fft::pad(i)].y);
    return 0;
  }
  if (!std::strcmp(mode, "c2cr")) {
    for (int i = 0; i < N; ++i) {
      double re, im;
      if (std::scanf("%lf %lf", &re, &im) != 2) return 1;
      at(i) = {re, im};
    }
    fft_regs<false>(buf, L);
    for (int i = 0; i < N; ++i) std::printf("%.17g\n%.17g\n", at(i).x, at(i).y);
  } else if (!std::strcmp(mode, "c2c") || !std::strcmp(mode, "ic2c")) {
    for (int i = 0; i < N; ++i) {
      double re, im;
      if (std::scanf("%lf %lf", &re, &im) != 2) return 1;
      at(i) = {re, im};
    }
    if (mode[0] == 'i')
      fft<true>(buf, L);
    else
      fft<false>(buf, L);
    for (int i = 0; i < N; ++i) std::printf("%.17g\n%.17g\n", at(i).x, at(i).y);
  } else if (!std::strcmp(mode, "r2c")) {
    for (int i = 0; i < N; ++i) {
      double a, b;
      if (std::scanf("%lf %lf", &a, &b) != 2) return 1;
      at(i) = {a, b};  // z[n] = x[2n] + i x[2n+1]
    }
    fft<false>(buf, L);
    for (int k = 0; k <= N; ++k) {
      const C z = at(k % N), zn = at((N - k) % N);
      const C X = gpn::fft::r2c_split(z, zn, wnf[k]);
      std::printf("%.17g\n%.17g\n", X.x, X.y);
    }
  } else if (!std::strcmp(mode, "c2r")) {
    std::vector<C> X(N + 1);
    for (int k = 0; k <= N; ++k)
      if (std::scanf("%lf %lf", &X[k].x, &X[k].y) != 2) return 1;
    for (int k = 0; k < N; ++k) at(k) = gpn::fft::c2r_merge(X[k], X[N - k], wnf[k]);
    fft<true>(buf, L);
    for (int n = 0; n < N; ++n) std::printf("%.17g\n%.17g\n", at(n).x, at(n).y);
  } else {
    return 1;
  }
  return 0;
}
