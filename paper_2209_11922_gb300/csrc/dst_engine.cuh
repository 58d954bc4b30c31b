// dst_engine.cuh - orthonormal DST-I of many pencils, as used by the fast solve of Section 4.
//
// The transform applied along one axis of length N (N-1 interior nodes) is
//     F_k = sqrt(2/N) * sum_{j=1}^{N-1} x_j sin(pi j k / N),  k = 1..N-1,
// i.e. S = sqrt(2/N) P with the sine matrix P of Section 4 (S is symmetric and S^2 = I, so the
// same routine is the forward transform and its inverse; Section 4 states the DST/iDST per axis).
//
// Two real pencils a, b are packed as one complex sequence c_j = a_j + i b_j and transformed by
// one complex FFT computed with Stockham passes whose butterflies (radix R <= 16 here) run in
// registers, with one shared-memory exchange per pass. Two variants:
//
// ODD (used for FP32): the odd extension z_j = c_j, z_{2N-j} = -c_j, z_0 = z_N = 0 of length
//   M = 2N has DFT Z_k = 2i sum_j c_j sin(pi j k / N) (kernel exp(+2 pi i j k / M)), so the outputs
//   are -i sc Z_k for k = 1..N-1 (sc = sqrt(2/N)/2). Rounding grows like log N only.
// RECURRENCE (used for FP64, half the FFT length, M = N):
//   1. y_j = sin(pi j/N)(c_j + c_{N-j}) + (c_j - c_{N-j})/2 for j = 1..N-1, y_0 = 0.
//   2. Z = length-N DFT of y.
//   3. With Y^a, Y^b the real DFTs separated from Z: F_{2k} = Im Y_k and
//      F_{2k+1} = F_{2k-1} + Re Y_k (F_1 = Re Y_0 / 2), i.e. even outputs are
//      (-i/2)(Z_k - Z_{N-k}) and odd outputs are half a prefix sum of G_0 = Z_0,
//      G_m = Z_m + Z_{N-m}; the prefix sum runs per thread then across lanes by warp shuffles.
//   The identities follow from splitting y into its even and odd parts about N/2. The prefix sum
//   lets rounding grow like sqrt(N/2) eps, which FP64 absorbs and FP32 does not.
//
// HARTLEY (periodic axes, FP32 and FP64, M = N): the orthonormal discrete Hartley transform
//     H_k = (1/sqrt(N)) sum_{j=0}^{N-1} x_j cas(2 pi j k / N),  cas t = cos t + sin t,  k = 0..N-1,
//   which is symmetric and its own inverse, and diagonalises the circulant A and B of the periodic
//   case because their eigenvalues depend on cos(2 pi k / N) only (modes k and N-k agree); it
//   stands in for the DFT / inverse DFT pair of Section 4's remarks on periodic boundaries with
//   real arithmetic throughout. The pair's length-N DFT Z (kernel exp(+2 pi i j k / N)) separates
//   into the two real sequences' DFTs, A_k = (Z_k + conj Z_{N-k})/2 and
//   B_k = (Z_k - conj Z_{N-k})/(2i), and H = Re + Im of each, so with z = Z_k, w = Z_{N-k}:
//     H^a_k = sc (z.x + w.x + z.y - w.y),  H^b_k = sc (z.y + w.y + w.x - z.x),  sc = 1/(2 sqrt(N)).
//   Every position 0..N-1 is data (no boundary slot).
//
// Layout: one pair occupies LP complex slots of shared memory; position j lives at
// j + j / PADG (one padding slot every PADG entries) so that the strided writes of the first pass
// hit distinct banks. Slot 0 holds position 0, which for the sine variants is the boundary node /
// mode 0 and is 0.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace etd {

template <class T> struct Cx { T x, y; };

template <class T> __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T> __device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return {s * a.x, s * a.y}; }
template <class T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __device__ __forceinline__ Cx<T> mul_i(Cx<T> a) { return {-a.y, a.x}; }

// cos(2 pi m / 96) for 0 <= m <= 24 (quarter wave), then by symmetry for any m >= 0.
__host__ __device__ constexpr double qcos96(int m) {
  switch (m) {
    case 0: return 1.0;
    case 1: return 0.9978589232386035;
    case 2: return 0.9914448613738104;
    case 3: return 0.9807852804032304;
    case 4: return 0.9659258262890683;
    case 5: return 0.9469301294951057;
    case 6: return 0.9238795325112867;
    case 7: return 0.8968727415326883;
    case 8: return 0.8660254037844386;
    case 9: return 0.8314696123025452;
    case 10: return 0.7933533402912352;
    case 11: return 0.7518398074789774;
    case 12: return 0.7071067811865476;
    case 13: return 0.6593458151000688;
    case 14: return 0.6087614290087207;
    case 15: return 0.5555702330196022;
    case 16: return 0.5;
    case 17: return 0.4422886902190013;
    case 18: return 0.3826834323650898;
    case 19: return 0.3214394653031616;
    case 20: return 0.25881904510252074;
    case 21: return 0.19509032201612828;
    case 22: return 0.1305261922200516;
    case 23: return 0.06540312923014306;
    default: return 0.0;  // m == 24
  }
}
__host__ __device__ constexpr double cos96(int m) {
  m %= 96;
  return m <= 24 ? qcos96(m) : m <= 48 ? -qcos96(48 - m) : m <= 72 ? -qcos96(m - 48) : qcos96(96 - m);
}
__host__ __device__ constexpr double sin96(int m) { return cos96((m % 96) + 72); }  // sin t = cos(t - pi/2)

// Compile-time loop: f(std::integral_constant<int, I>) for I = B..E-1.
template <int B, int E, class F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// v * exp(2 pi i M / 96) with M a template constant: the trivial factors are exact and the others
// are literal constants.
template <class T, int M> __device__ __forceinline__ Cx<T> twmul96(Cx<T> v) {
  constexpr int m = M % 96;
  if constexpr (m == 0) return v;
  else if constexpr (m == 24) return {-v.y, v.x};
  else if constexpr (m == 48) return {-v.x, -v.y};
  else if constexpr (m == 72) return {v.y, -v.x};
  else {
    constexpr T c = (T)cos96(m), s = (T)sin96(m);
    return {c * v.x - s * v.y, c * v.y + s * v.x};
  }
}

// In-register DFT of length R with kernel exp(+2 pi i r k / R), natural order in and out.
template <class T, int R> struct Dft {
  static_assert(96 % R == 0, "radix must divide 96");
  static constexpr int F = (R % 4 == 0) ? 4 : (R % 2 == 0 ? 2 : 3);
  static constexpr int Q = R / F;
  static __device__ __forceinline__ void run(Cx<T>* x);
};
template <class T> struct Dft<T, 1> { static __device__ __forceinline__ void run(Cx<T>*) {} };
template <class T> struct Dft<T, 2> {
  static __device__ __forceinline__ void run(Cx<T>* x) {
    const Cx<T> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  }
};
template <class T> struct Dft<T, 3> {
  static __device__ __forceinline__ void run(Cx<T>* x) {
    const Cx<T> s = x[1] + x[2], d = x[1] - x[2];
    const Cx<T> t = x[0] - T(0.5) * s;
    const Cx<T> u = mul_i(T(0.86602540378443864676) * d);
    x[0] = x[0] + s;
    x[1] = t + u;
    x[2] = t - u;
  }
};
template <class T> struct Dft<T, 4> {
  static __device__ __forceinline__ void run(Cx<T>* x) {
    const Cx<T> a0 = x[0] + x[2], a1 = x[0] - x[2], b0 = x[1] + x[3], b1 = mul_i(x[1] - x[3]);
    x[0] = a0 + b0;
    x[2] = a0 - b0;
    x[1] = a1 + b1;
    x[3] = a1 - b1;
  }
};
template <class T, int R>
__device__ __forceinline__ void Dft<T, R>::run(Cx<T>* x) {
  Cx<T> y[F][Q];
#pragma unroll
  for (int s = 0; s < F; ++s)
#pragma unroll
    for (int q = 0; q < Q; ++q) y[s][q] = x[F * q + s];
#pragma unroll
  for (int s = 0; s < F; ++s) Dft<T, Q>::run(y[s]);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    Cx<T> a[F];
    static_for<0, F>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      a[s] = twmul96<T, (96 / R) * s * k>(y[s][k]);
    });
    Dft<T, F>::run(a);
#pragma unroll
    for (int t = 0; t < F; ++t) x[k + Q * t] = a[t];
  });
}

// Per-(type, N) pass plan: FFT length M, radices of the Stockham passes, threads per pair (TPP).
// A thread holds at most 32 (FP32) / 16 (FP64) complex values in a pass; the last radix of an ODD
// plan is even so that the outputs k < N are exactly the butterfly outputs r < R/2.
template <int... Rs> struct Radices {};
template <class T, int N, bool ODD> struct FftPlan;
// Transform variant of a kernel (template argument VAR): the two DST-I forms and the Hartley form.
// The Hartley variant runs the recurrence variant's length-N FFT plan.
enum Variant : int { V_REC = 0, V_ODD = 1, V_HART = 2 };
#define ETD_PLAN(TYPE, NN, ODD_, TPP_, ...)                \
  template <> struct FftPlan<TYPE, NN, ODD_> {             \
    static constexpr bool ODD = ODD_;                      \
    static constexpr int M = ODD_ ? 2 * NN : NN;           \
    static constexpr int TPP = TPP_;                       \
    using R = Radices<__VA_ARGS__>;                        \
  };
// FP32: odd extension, M = 2N
ETD_PLAN(float, 4, true, 2, 4, 2)
ETD_PLAN(float, 8, true, 4, 4, 4)
ETD_PLAN(float, 16, true, 8, 8, 4)
ETD_PLAN(float, 32, true, 8, 8, 8)
ETD_PLAN(float, 64, true, 16, 16, 8)
ETD_PLAN(float, 128, true, 16, 16, 16)
ETD_PLAN(float, 256, true, 64, 8, 8, 8)
ETD_PLAN(float, 512, true, 128, 16, 8, 8)
ETD_PLAN(float, 1024, true, 128, 16, 8, 16)
ETD_PLAN(float, 2048, true, 256, 16, 16, 16)
ETD_PLAN(float, 6, true, 4, 3, 4)
ETD_PLAN(float, 12, true, 8, 3, 8)
ETD_PLAN(float, 24, true, 4, 12, 4)
ETD_PLAN(float, 48, true, 8, 12, 8)
ETD_PLAN(float, 96, true, 16, 12, 16)
ETD_PLAN(float, 192, true, 64, 6, 4, 16)
ETD_PLAN(float, 384, true, 64, 12, 4, 16)
ETD_PLAN(float, 768, true, 128, 12, 8, 16)
ETD_PLAN(float, 1536, true, 256, 12, 16, 16)
// FP32 and FP64: recurrence, M = N
ETD_PLAN(float, 4, false, 1, 4)
ETD_PLAN(float, 8, false, 2, 4, 2)
ETD_PLAN(float, 16, false, 4, 4, 4)
ETD_PLAN(float, 32, false, 4, 8, 4)
ETD_PLAN(float, 64, false, 8, 8, 8)
ETD_PLAN(float, 128, false, 8, 16, 8)
ETD_PLAN(float, 256, false, 16, 16, 16)
ETD_PLAN(float, 512, false, 64, 8, 8, 8)
ETD_PLAN(float, 1024, false, 128, 8, 8, 16)
ETD_PLAN(float, 2048, false, 128, 16, 8, 16)
ETD_PLAN(float, 6, false, 1, 6)
ETD_PLAN(float, 12, false, 2, 4, 3)
ETD_PLAN(float, 24, false, 4, 8, 3)
ETD_PLAN(float, 48, false, 4, 12, 4)
ETD_PLAN(float, 96, false, 16, 4, 3, 8)
ETD_PLAN(float, 192, false, 16, 16, 12)
ETD_PLAN(float, 384, false, 32, 8, 3, 16)
ETD_PLAN(float, 768, false, 64, 16, 3, 16)
ETD_PLAN(float, 1536, false, 128, 16, 6, 16)
ETD_PLAN(double, 4, false, 1, 4)
ETD_PLAN(double, 8, false, 2, 4, 2)
ETD_PLAN(double, 16, false, 4, 4, 4)
ETD_PLAN(double, 32, false, 4, 8, 4)
ETD_PLAN(double, 64, false, 8, 8, 8)
ETD_PLAN(double, 128, false, 8, 16, 8)
ETD_PLAN(double, 256, false, 16, 16, 16)
ETD_PLAN(double, 512, false, 32, 8, 8, 8)
ETD_PLAN(double, 1024, false, 64, 16, 8, 8)
ETD_PLAN(double, 2048, false, 128, 16, 16, 8)
ETD_PLAN(double, 6, false, 1, 6)
ETD_PLAN(double, 12, false, 2, 4, 3)
ETD_PLAN(double, 24, false, 4, 8, 3)
ETD_PLAN(double, 48, false, 4, 12, 4)
ETD_PLAN(double, 96, false, 8, 12, 8)
ETD_PLAN(double, 192, false, 16, 12, 16)
ETD_PLAN(double, 384, false, 32, 8, 3, 16)
ETD_PLAN(double, 768, false, 64, 16, 3, 16)
ETD_PLAN(double, 1536, false, 128, 16, 6, 16)
#undef ETD_PLAN

template <class L> struct FirstRadix;
template <int R0, int... Rs> struct FirstRadix<Radices<R0, Rs...>> { static constexpr int value = R0; };

// Twiddle tables: for every pass after the first (NS > 1) the factors w_M^{k r M/(NS R)},
// k = jj mod NS < NS, r = 1..R-1, are stored r-major at [(r-1)*NS + k], passes back to back, so
// the lanes of a warp (consecutive jj) read consecutive entries. TwOffset gives a pass's start.
template <int NS, int... Rs> struct TwSize { static constexpr int value = 0; };
template <int NS, int R, int... Rest> struct TwSize<NS, R, Rest...> {
  static constexpr int value = (NS > 1 ? (R - 1) * NS : 0) + TwSize<NS * R, Rest...>::value;
};
template <class L> struct TwiddleCount;
template <int... Rs> struct TwiddleCount<Radices<Rs...>> { static constexpr int value = TwSize<1, Rs...>::value; };

template <class T, int N, int VAR> struct PairLayout {
  using Plan = FftPlan<T, N, VAR == V_ODD>;
  static constexpr bool ODD = Plan::ODD;
  static constexpr bool HART = VAR == V_HART;
  static constexpr int M = Plan::M;
  static constexpr int TPP = Plan::TPP;
  static constexpr int PADG = FirstRadix<typename Plan::R>::value;
  static constexpr int LP = M + M / PADG + 1;  // minimum complex slots per pair
  static constexpr int TWN = TwiddleCount<typename Plan::R>::value;  // twiddle table entries
  static __device__ __forceinline__ int at(int j) { return j + j / PADG; }
  // at(j0 + k*TPP) for 0 <= j0 < TPP, linear in k when PADG divides TPP
  static __device__ __forceinline__ int at_stride(int atj0, int j0, int k) {
    if constexpr (TPP % PADG == 0) return atj0 + k * (TPP + TPP / PADG);
    else return at(j0 + k * TPP);
  }
};

// ---------------------------------------------------------------------------------------------
// Stockham passes over the length-M sequence. Pass with radix R after Ns points are combined:
// butterfly jj reads positions jj + r*M/R, twiddles by w_M^{(jj mod Ns) r M/(Ns R)}, and writes
// (jj/Ns)*Ns*R + (jj mod Ns) + r*Ns. In place: all reads, barrier, all writes, barrier.
// The first pass folds in the input map of the variant (odd extension or the y_j of the
// recurrence); the last pass of the ODD variant writes only k < N, already scaled by -i sc.
// Nodal reaction f(u) = flin u + fcub u^3 applied to both packed pencils as the first pass reads
// them (the logarithmic term of the Flory-Huggins reaction is applied by the pass kernel itself,
// outside the butterfly code).
template <class T> struct React {
  bool on;
  T flin, fcub;
  __device__ __forceinline__ Cx<T> operator()(Cx<T> c) const {
    return on ? Cx<T>{c.x * (flin + fcub * c.x * c.x), c.y * (flin + fcub * c.y * c.y)} : c;
  }
};

template <class T, int N, int VAR, int NB, int NS, bool FIRST, int R, int... Rest>
__device__ __forceinline__ void stockham(Cx<T>* const (&bps)[NB], const Cx<T>* __restrict__ tw,
                                         const T* __restrict__ sn, int l, T sc, React<T> rx) {
  // tw points at this pass's table (unused when NS == 1); the first pass applies rx to its input.
  // NB independent pairs (one per buffer) go through the pass together, sharing its barriers.
  using L = PairLayout<T, N, VAR>;
  constexpr int M = L::M;
  constexpr int TPP = L::TPP;
  constexpr int TP = M / R;
  constexpr int QN = (TP + TPP - 1) / TPP;
  constexpr bool LAST = sizeof...(Rest) == 0;
  Cx<T> v[NB][QN][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    Cx<T>* __restrict__ bp = bps[b];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int jj = l + TPP * q;
      if (TP % TPP == 0 || jj < TP) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int idx = jj + r * TP;
          Cx<T> xv;
          if constexpr (FIRST && L::ODD) {
            if (idx == 0 || idx == N) {
              xv = {T(0), T(0)};
            } else if (idx < N) {
              xv = rx(bp[L::at(idx)]);
            } else {
              const Cx<T> c = rx(bp[L::at(M - idx)]);
              xv = {-c.x, -c.y};
            }
          } else if constexpr (FIRST && L::HART) {
            xv = rx(bp[L::at(idx)]);
          } else if constexpr (FIRST) {
            if (idx == 0) {
              xv = {T(0), T(0)};
            } else {
              const Cx<T> c = rx(bp[L::at(idx)]), d = rx(bp[L::at(N - idx)]);
              const T s = sn[idx];
              xv = s * (c + d) + T(0.5) * (c - d);
            }
          } else {
            xv = bp[L::at(idx)];
          }
          if (NS > 1 && r > 0) xv = cmul(xv, tw[(r - 1) * NS + (jj % NS)]);
          v[b][q][r] = xv;
        }
        Dft<T, R>::run(v[b][q]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    Cx<T>* __restrict__ bp = bps[b];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int jj = l + TPP * q;
      if (TP % TPP == 0 || jj < TP) {
        const int base = (jj / NS) * NS * R + (jj % NS);
        if constexpr (LAST && L::ODD) {
          static_assert(R % 2 == 0 && NS * R == M, "last ODD radix must be even");
#pragma unroll
          for (int r = 0; r < R / 2; ++r) {   // k = jj + r*NS < N
            const Cx<T> z = v[b][q][r];
            const int k = base + r * NS;
            bp[L::at(k)] = (k == 0) ? Cx<T>{T(0), T(0)} : Cx<T>{sc * z.y, -sc * z.x};
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) bp[L::at(base + r * NS)] = v[b][q][r];
        }
      }
    }
  }
  __syncthreads();
  if constexpr (!LAST)
    stockham<T, N, VAR, NB, NS * R, false, Rest...>(bps, tw + (NS > 1 ? (R - 1) * NS : 0), sn, l, sc, rx);
}

template <class T, int N, int VAR, int NB, int... Rs>
__device__ __forceinline__ void run_fft(Cx<T>* const (&bps)[NB], const Cx<T>* tw, const T* sn, int l, T sc,
                                        React<T> rx, Radices<Rs...>) {
  stockham<T, N, VAR, NB, 1, true, Rs...>(bps, tw, sn, l, sc, rx);
}

// `mask` names the lanes of the warp that exist (a CTA may have fewer than 32 threads).
template <class T>
__device__ __forceinline__ Cx<T> shfl_up_cx(unsigned mask, Cx<T> v, int d, int width) {
  return {__shfl_up_sync(mask, v.x, d, width), __shfl_up_sync(mask, v.y, d, width)};
}

// Full orthonormal DST-I (Hartley variant: DHT) of NB independent pairs (one per buffer bps[b]), in
// place: on return positions 0..N-1 of each hold the result (DST: position 0 = 0). sc = sqrt(2/N)/2
// (DHT: 1/(2 sqrt(N))). tw holds the
// per-pass twiddle tables, sn = sin(pi j / N) (recurrence only). scrs[b] is shared scratch of
// TPP/32 complex per pair (recurrence, TPP > 32). With rx.on the input is first mapped through the
// nodal reaction (fused into the first pass). Running two transforms together halves the number
// of barrier-separated phases they cost.
template <class T, int N, int VAR, int NB>
__device__ __forceinline__ void dst_pairs(Cx<T>* const (&bps)[NB], const Cx<T>* __restrict__ tw,
                                          const T* __restrict__ sn, int l, Cx<T>* const (&scrs)[NB], T sc,
                                          React<T> rx = React<T>{false, T(0), T(0)}) {
  using L = PairLayout<T, N, VAR>;
  run_fft<T, N, VAR, NB>(bps, tw, sn, l, sc, rx, typename L::Plan::R{});
  if constexpr (L::HART) {
    // each thread owns the position pairs (k, N-k), k = l, l + TPP, .. <= N/2: no barrier between
    // its reads and writes
    constexpr int TPP = L::TPP;
    constexpr int C = (N / 2 + 1 + TPP - 1) / TPP;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      Cx<T>* __restrict__ bp = bps[b];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int k = l + i * TPP;
        if (k <= N / 2) {
          const int m = k == 0 ? 0 : N - k;
          const Cx<T> z = bp[L::at(k)], w = bp[L::at(m)];
          bp[L::at(k)] = Cx<T>{sc * (z.x + w.x + z.y - w.y), sc * (z.y + w.y + w.x - z.x)};
          if (m != k) bp[L::at(m)] = Cx<T>{sc * (w.x + z.x + w.y - z.y), sc * (w.y + z.y + z.x - w.x)};
        }
      }
    }
    __syncthreads();
  } else if constexpr (!L::ODD) {
    constexpr int TPP = L::TPP;
    constexpr int C = (N / 2) / TPP;
    static_assert(C * TPP == N / 2, "N/2 must be a multiple of the threads per pair");
    constexpr int W = TPP < 32 ? TPP : 32;
    const int ls = l % W;
    const unsigned mask = __activemask();  // every thread of the CTA reaches this point converged
    Cx<T> g[NB][C], e[NB][C], off[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      Cx<T>* __restrict__ bp = bps[b];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int m = l * C + i;
        const Cx<T> zm = bp[L::at(m)];
        if (m == 0) {
          g[b][i] = zm;
          e[b][i] = {T(0), T(0)};
        } else {
          const Cx<T> zn = bp[L::at(N - m)];
          g[b][i] = zm + zn;
          const Cx<T> d = zm - zn;
          e[b][i] = {d.y, -d.x};
        }
        if (i > 0) g[b][i] = g[b][i] + g[b][i - 1];
      }
      // exclusive offset of this lane's chunk within the pair
      const Cx<T> tot = g[b][C - 1];
      Cx<T> inc = tot;
#pragma unroll
      for (int d = 1; d < W; d <<= 1) {
        const Cx<T> t = shfl_up_cx(mask, inc, d, W);
        if (ls >= d) inc = inc + t;
      }
      if constexpr (TPP > 32) {
        if (ls == 31) scrs[b][l / 32] = inc;
      }
      off[b] = inc - tot;
    }
    __syncthreads();
    if constexpr (TPP > 32) {
      constexpr int NW = TPP / 32;
      const int w = l / 32;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < NW - 1; ++k)
          if (k < w) off[b] = off[b] + scrs[b][k];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      Cx<T>* __restrict__ bp = bps[b];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int m = l * C + i;
        bp[L::at(2 * m)] = (m == 0) ? Cx<T>{T(0), T(0)} : sc * e[b][i];
        bp[L::at(2 * m + 1)] = sc * (g[b][i] + off[b]);
      }
    }
    __syncthreads();
  }
}

template <class T, int N, int VAR>
__device__ __forceinline__ void dst_pair(Cx<T>* bp, const Cx<T>* __restrict__ tw, const T* __restrict__ sn, int l,
                                         Cx<T>* scr, T sc, React<T> rx = React<T>{false, T(0), T(0)}) {
  Cx<T>* const bps[1] = {bp};
  Cx<T>* const scrs[1] = {scr};
  dst_pairs<T, N, VAR, 1>(bps, tw, sn, l, scrs, sc, rx);
}

// Pointwise epilogue over positions 0..N-1 of one pair: bp[j] = epi(j, bp[j]). The loop is kept
// rolled so that the epilogue's code appears once in the kernel.
template <class T, int N, int VAR, class Epi>
__device__ __forceinline__ void epilogue_pair(Cx<T>* __restrict__ bp, int l, Epi&& epi) {
  using L = PairLayout<T, N, VAR>;
#pragma unroll 1
  for (int j = l; j < N; j += L::TPP) bp[L::at(j)] = epi(j, bp[L::at(j)]);
  __syncthreads();
}

}  // namespace etd
