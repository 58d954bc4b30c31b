// split_dst.cuh - FP32 orthonormal DST-I of pencil pairs of length N = 1024 by a split-radix
// decomposition whose sub-transforms each fit in one warp.
//
// The transform is S = sqrt(2/N) P with the sine matrix P of Section 4 (S^2 = I: the same routine is the
// forward transform and its inverse). With x_0 = x_N = 0 and S_k = sum_{j=1}^{N-1} x_j sin(pi j k/N), the
// output index is split by parity, using sin(pi (N-j) k / N) = -(-1)^k sin(pi j k / N):
//   k = 2m+1:  S_k = sum_{j=1}^{N/2} b1_j sin(pi j (2m+1) / N),   b1_j = x_j + x_{N-j} (j < N/2), b1_{N/2} = x_{N/2},
//              a DST-III of length N/2;
//   k = 2m:    S_k = sum_{j=1}^{N/2-1} a1_j sin(pi j m / (N/2)),   a1_j = x_j - x_{N-j},  a DST-I of length N/2,
// and the second half once more: its odd outputs (k = 2 mod 4) are a DST-III of length N/4 of
// b2_j = a1_j + a1_{N/2-j} (b2_{N/4} = a1_{N/4}), its even outputs (k = 0 mod 4) a DST-I of length N/4 of
// a2_j = a1_j - a1_{N/2-j}.
// A DST-III T_m = sum_{j=1}^{M} b_j sin(pi j (2m+1) / (2M)) is one complex FFT of length M between a
// pre-twiddle and a permutation (it is (-1)^m times the DCT-III of the reversed sequence, computed as the
// inverse of the even/odd reordering of a DCT-II):
//   W_k = (1/2) e^{i pi k / (2M)} (b_{M-k} - i b_k)   (k = 0 gives W_0 = b_M),
//   v_n = sum_k W_k e^{2 pi i n k / M},   T_{2n} = v_n,   T_{2n+1} = -v_{M-1-n}.
// The DST-I of length N/4 is read off the FFT of the odd extension of a2 (length N/2), Z_p = 2i sum_j a2_j
// sin(pi j p / (N/4)). All maps are linear over the complex numbers, so two real pencils a, b travel as one
// complex sequence c = a + i b.
//
// For N = 1024 the three FFTs have 512 (A: DST-III of b1), 256 (B: DST-III of b2) and 512 (C: odd extension
// of a2) points, 1280 in all, against 2048 for the odd extension of the whole pencil. Each runs within one
// warp: 16 points per lane, a radix-16 butterfly in registers, a twiddle, one warp-local transpose through
// shared memory (__syncwarp only), a second radix-16 butterfly and, for 512 points, a radix-2 step between
// the half-warps by shuffles. Roles A and C each take a warp per pair and read the four inputs x_k,
// x_{N-k}, x_{N/2-k}, x_{N/2+k} that each FFT input combines; B takes one warp for two pairs (a half-warp
// each, eight inputs per point). Rounding grows like log N.
//
// Pair buffer layout: position j (0..N) of a pair lives at slot j + j/16. Any 16 consecutive positions
// then sit on distinct banks, the strided output positions of the three FFTs (stride 4 or 8) too, and every
// gather and scatter address is a per-lane base plus a compile-time multiple of the register index.
// Positions 0 and N hold 0 and are never written by a transform.
#pragma once
#include <cuda_runtime.h>

#include "dst_engine.cuh"

namespace etd {

constexpr int SPLIT_N = 1024;
constexpr int SPLIT_LPS = 1092;       // complex slots per pair buffer: > slot(N) = 1088, = 4 (mod 16) so that
                                      // the buffers of consecutive pairs start on staggered banks
// twiddle table of a split axis (complex, FP64 values rounded once to FP32), in this order:
constexpr int SPLIT_PREA = 0;         // [512]   (1/2) sqrt(2/N) e^{i pi k / N}, k < 512
constexpr int SPLIT_TWA = 512;        // [15][32] e^{2 pi i n k / 512}, n = 1..15, k < 32
constexpr int SPLIT_PREB = 992;       // [256]   (1/2) sqrt(2/N) e^{i pi k / (N/2)}, k < 256
constexpr int SPLIT_TWB = 1248;       // [15][16] e^{2 pi i n k / 256}, n = 1..15, k < 16
constexpr int SPLIT_TWN = 1488;
constexpr int SPLIT_SCR = 544;        // transpose scratch per warp (complex): 16 x 33, or 2 x 16 x 17

__host__ __device__ constexpr int sslot(int j) { return j + (j >> 4); }

using Cf = Cx<float>;

__device__ __forceinline__ Cf shfl_xor_cx(Cf v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

// 256-point FFT of v[r] = W[hl + 16 r] across a half-warp (hl = lane & 15, its own scratch). On return
// v[n1] = out[hl + 16 n1].
__device__ __forceinline__ void fft256_half(Cf (&v)[16], const Cf* __restrict__ tab, Cf* __restrict__ scr, int hl) {
#pragma unroll 1
  for (int st = 0; st < 2; ++st) {
    Dft<float, 16>::run(v);
    if (st == 0) {
#pragma unroll
      for (int n = 1; n < 16; ++n) v[n] = cmul(v[n], tab[SPLIT_TWB + (n - 1) * 16 + hl]);   // e^{2 pi i n2 k1 / 256}
      __syncwarp();
#pragma unroll
      for (int n = 0; n < 16; ++n) scr[n * 17 + hl] = v[n];
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = scr[hl * 17 + k];
    }
  }
}

// 512-point FFT of v[r] = W[lane + 32 r] across one warp (kernel e^{+2 pi i n k / 512}). On return lane
// (a = lane >> 4, n2 = lane & 15) holds out[n2 + 16 c] for a = 0 and -out[n2 + 16 c + 256] for a = 1 in
// v[c]. (512 = 16 x 32: k = k1 + 32 k2, n = n2 + 16 n1; the 32-point stage is 16 x 2 with k1 = a + 2 b.)
__device__ __forceinline__ void fft512_warp(Cf (&v)[16], const Cf* __restrict__ tab, Cf* __restrict__ scr, int lane) {
  const int n2 = lane & 15, a = lane >> 4;
#pragma unroll 1
  for (int st = 0; st < 2; ++st) {
    Dft<float, 16>::run(v);
    if (st == 0) {
#pragma unroll
      for (int n = 1; n < 16; ++n) v[n] = cmul(v[n], tab[SPLIT_TWA + (n - 1) * 32 + lane]);   // e^{2 pi i n2 k1 / 512}
      __syncwarp();
#pragma unroll
      for (int n = 0; n < 16; ++n) scr[n * 33 + lane] = v[n];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < 16; ++b) v[b] = scr[n2 * 33 + a + 2 * b];
    }
  }
  if (a) {
    static_for<1, 16>([&](auto cc) {
      constexpr int c = decltype(cc)::value;
      v[c] = twmul96<float, 3 * c>(v[c]);                              // e^{2 pi i c a / 32}
    });
  }
  const float s = a ? -1.f : 1.f;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const Cf o = shfl_xor_cx(v[c], 16);
    v[c] = Cf{fmaf(s, o.x, v[c].x), fmaf(s, o.y, v[c].y)};
  }
}

// One DST-I of the two pairs of a group, in place in their buffers x0 (pair 0) and x1 (pair 1), by the
// group's five warps: role 0/1 A of pair 0/1, 2/3 C of pair 0/1, 4 B of both (lanes 0-15 pair 0, 16-31
// pair 1). Every thread of the CTA calls it: it holds two CTA barriers (after the gathers and FFTs, after
// the scatters); warps with active = false take part in the barriers only. With react the written values
// are mapped through f(u) = fl u + fc u^3 (the transform is then an inverse one whose outputs are nodal
// values). hsc = sqrt(2/N)/2 scales role C; A and B carry the scale in their pre-twiddles.
__device__ __forceinline__ void split_dst_group(int role, int lane, Cf* __restrict__ x0, Cf* __restrict__ x1,
                                                const Cf* __restrict__ tab, Cf* __restrict__ scr, bool active,
                                                bool react, float fl, float fc, float hsc) {
  Cf v[16];
  Cf* const x = (role == 1 || role == 3) ? x1 : (role == 4 ? (lane < 16 ? x0 : x1) : x0);
  if (active) {
    if (role == 4) {
      // W_k = pre_k (b2_{256-k} - i b2_k), k = hl + 16 r: slot(k) = hl + 17 r, slot(N - k) = gm - 17 r
      const int hl = lane & 15, gm = 1088 - hl - (hl > 0 ? 1 : 0);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int u = hl + 17 * r, d = gm - 17 * r;
        const Cf b2k = (x[u] - x[d]) + (x[d - 544] - x[u + 544]);             // k, N-k, N/2-k, N/2+k
        const Cf b2m = (x[d - 816] - x[u + 816]) + (x[u + 272] - x[d - 272]);  // 256-k, 768+k, 256+k, 768-k
        v[r] = cmul(Cf{b2m.x + b2k.y, b2m.y - b2k.x}, tab[SPLIT_PREB + hl + 16 * r]);
      }
      fft256_half(v, tab, scr + (lane >> 4) * 272, hl);
    } else {
      // k = lane + 32 r: slot(k) = g0 + 34 r, slot(N - k) = gm - 34 r, slot(N/2 -+ k) = those -+ 544
      const int g0 = lane + (lane >> 4), gm = 1088 - lane - ((lane + 15) >> 4);
      if (role < 2) {      // A: W_k = pre_k (b1_{512-k} - i b1_k)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int u = g0 + 34 * r, d = gm - 34 * r;
          const Cf bk = x[u] + x[d], bm = x[d - 544] + x[u + 544];
          v[r] = cmul(Cf{bm.x + bk.y, bm.y - bk.x}, tab[SPLIT_PREA + lane + 32 * r]);
        }
      } else {             // C: z_k = a2_k extended oddly
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int u = g0 + 34 * r, d = gm - 34 * r;
          v[r] = (x[u] - x[d]) - (x[d - 544] - x[u + 544]);
        }
      }
      fft512_warp(v, tab, scr, lane);
    }
  }
  __syncthreads();
  if (active) {
    auto put = [&](int s, Cf z) {
      if (react) z = Cf{z.x * (fl + fc * z.x * z.x), z.y * (fl + fc * z.y * z.y)};
      x[s] = z;
    };
    const int n2 = lane & 15;
    const bool hi = lane >= 16;
    if (role < 2) {        // A: a = 0 -> position 4n+1, a = 1 -> 4(511-n)+3, n = n2 + 16 c
      const int sb = hi ? 1086 - 4 * n2 - (n2 >> 2) : 4 * n2 + 1 + (n2 >> 2), ss = hi ? -68 : 68;
#pragma unroll
      for (int c = 0; c < 16; ++c) put(sb + ss * c, v[c]);
    } else if (role < 4) { // C: position 4p, p = n2 + 16 c in 1..255 (lanes a = 0): S_{4p} = -i Z_p / 2
      if (!hi) {
        const int cb = 4 * n2 + (n2 >> 2);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c > 0 || n2 > 0) put(cb + 68 * c, Cf{hsc * v[c].y, -hsc * v[c].x});
      }
    } else {               // B: position 8n + 2 (n = hl + 16 c < 128), 2046 - 8n (n >= 128, negated)
      const int sb = 8 * n2 + 2 + (n2 >> 1), sb2 = 1085 - 8 * n2 - (n2 >> 1);
#pragma unroll
      for (int c = 0; c < 8; ++c) put(sb + 136 * c, v[c]);
#pragma unroll
      for (int c = 8; c < 16; ++c) put(sb2 - 136 * (c - 8), Cf{-v[c].x, -v[c].y});
    }
  }
  __syncthreads();
}

}  // namespace etd
