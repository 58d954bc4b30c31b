// sno_kernels.cuh - kernels of the spectral neural operator (the learned coarse propagator of the
// Parareal loop) and its training: a strided batched FP32 GEMM with fused epilogues, elementwise
// maps (lift, GELU gradient, loss gradient), batch reductions and the Adam update.
//
// Operator (per field of an N x N mesh, n = N - 1 interior nodes per axis, C channels, M x M
// retained sine modes S_M[p][j] = sqrt(2/N) sin((p+1)(j+1) pi / N), L layers):
//   h_0 = lift(u, a);  per layer: hh = bf(S_M h S_M^T); gh[o] = sum_c bf(Wm[p,q,o,c]) hh[c];
//   z = S_M^T gh S_M + Wp h + bp;  h' = gelu(z);   u_hat = u + Wq . h_L + bq,
// with bf = round to bfloat16 and a = (ln D - ln 1e-3) / ln 100.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace etd {
namespace sno {

// round-to-nearest-even to bfloat16, kept in an fp32 register
__device__ __forceinline__ float bf16_round(float x) {
  uint32_t b = __float_as_uint(x);
  b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
  return __uint_as_float(b);
}
// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

enum GemmEpiKind : int {
  SG_NONE = 0,        // C = alpha acc + beta C
  SG_BIAS = 1,        // ... + bias[i]
  SG_BIAS_GELU = 2,   // ... + bias[i] -> C, gelu of it -> C2
  SG_RESID = 3,       // ... + R[b][i][j] (+ bias[i] when bias is given)
};

// C[b][i][j] = alpha sum_k A[b][i][k] B[b][k][j] (+ beta C) (+ epilogue), every operand addressed
// by (row, column, batch) element strides, so transposes and broadcasts are strides.
struct SGemm {
  int M, N, K, batch;
  const float* A; long long a_rs, a_cs, a_bs;
  const float* B; long long b_rs, b_cs, b_bs;
  float* C; long long c_rs, c_cs, c_bs;
  float alpha, beta;
  int round_a, round_b, round_c;   // bf16 rounding of A, B on load, of the result on store
  int epi;
  const float* bias;               // [M] (SG_BIAS, SG_BIAS_GELU)
  float* C2;                       // gelu(C) with C's strides (SG_BIAS_GELU)
  const float* R;                  // with C's strides (SG_RESID; bias[i] is added too when given)
  int ksplit;                      // >1: blockIdx.z = batch * ksplit + s sums K range s into C + s * c_ss
  long long c_ss;
};

constexpr int SG_BK = 16;

// Tile BM x BN per CTA of 256 threads (16 x 16); thread (tx, ty) owns rows 2 ty + 32 a + {0, 1} and
// columns 2 tx + 32 b + {0, 1} (pairs read as float2 from shared memory, and a warp's stores of one
// row cover 128 contiguous bytes); K in steps of 16 through shared memory. Operand loads walk the
// contiguous index of each operand. Shapes: 64 x 64 in general, 128 x 128 for large square
// outputs, 32 x 128 / 128 x 32 for the skinny ones (C = 32 channels, M = 24 modes).
template <int BM, int BN>
__global__ void __launch_bounds__(256, 2) sgemm_kernel(const SGemm g) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ __align__(16) float As[SG_BK][BM + 4];
  __shared__ __align__(16) float Bs[SG_BK][BN + 4];
  const int ks = g.ksplit > 1 ? g.ksplit : 1;
  const int bz = blockIdx.z / ks, sk = blockIdx.z % ks;
  const int kc = ((g.K + ks - 1) / ks + SG_BK - 1) / SG_BK * SG_BK;   // K range of this split
  const int kbeg = sk * kc, kend = min(g.K, kbeg + kc);
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const float* A = g.A + bz * g.a_bs;
  const float* B = g.B + bz * g.b_bs;
  float acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.f;
  const bool a_kfast = g.a_cs == 1 || g.a_rs != 1;
  const bool b_jfast = g.b_cs == 1 || g.b_rs != 1;
  for (int k0 = kbeg; k0 < kend; k0 += SG_BK) {
#pragma unroll
    for (int e = t; e < BM * SG_BK; e += 256) {
      int ii, kk;
      if (a_kfast) { ii = e / SG_BK; kk = e % SG_BK; }
      else { ii = e % BM; kk = e / BM; }
      const int gi = i0 + ii, gk = k0 + kk;
      const float v = (gi < g.M && gk < kend) ? A[gi * g.a_rs + gk * g.a_cs] : 0.f;
      As[kk][ii] = g.round_a ? bf16_round(v) : v;
    }
#pragma unroll
    for (int e = t; e < BN * SG_BK; e += 256) {
      int jj, kb;
      if (b_jfast) { jj = e % BN; kb = e / BN; }
      else { jj = e / SG_BK; kb = e % SG_BK; }
      const int gj = j0 + jj, gkb = k0 + kb;
      const float w = (gj < g.N && gkb < kend) ? B[gkb * g.b_rs + gj * g.b_cs] : 0.f;
      Bs[kb][jj] = g.round_b ? bf16_round(w) : w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int x = 0; x < TM; x += 2) {
        const float2 v = *reinterpret_cast<const float2*>(&As[kk][2 * ty + 16 * x]);
        a[x] = v.x;
        a[x + 1] = v.y;
      }
#pragma unroll
      for (int y = 0; y < TN; y += 2) {
        const float2 v = *reinterpret_cast<const float2*>(&Bs[kk][2 * tx + 16 * y]);
        b[y] = v.x;
        b[y + 1] = v.y;
      }
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int i = i0 + 2 * ty + 16 * (x & ~1) + (x & 1);
    if (i >= g.M) continue;
#pragma unroll
    for (int y = 0; y < TN; ++y) {
      const int j = j0 + 2 * tx + 16 * (y & ~1) + (y & 1);
      if (j >= g.N) continue;
      const long long ci = bz * g.c_bs + i * g.c_rs + j * g.c_cs;
      const long long co = ci + (ks > 1 ? sk * g.c_ss : 0);
      float v = g.alpha * acc[x][y];
      if (g.beta != 0.f) v += g.beta * g.C[co];
      if (g.epi == SG_BIAS || g.epi == SG_BIAS_GELU) v += g.bias[i];
      if (g.epi == SG_RESID) v += g.R[ci] + (g.bias ? g.bias[i] : 0.f);
      if (g.round_c) v = bf16_round(v);
      g.C[co] = v;
      if (g.epi == SG_BIAS_GELU) g.C2[ci] = gelu(v);
    }
  }
}

// h0[b][c][i] = Wl[c][0] u[b][i] + Wl[c][1] a[b] + bl[c]; blockIdx.y = b * C + c
__global__ void lift_kernel(const float* __restrict__ u, const float* __restrict__ a, const float* __restrict__ Wl,
                            const float* __restrict__ bl, float* __restrict__ h, int B, int C, long long npix) {
  const int bc = blockIdx.y, b = bc / C, c = bc - b * C;
  const float w0 = Wl[2 * c], off = Wl[2 * c + 1] * a[b] + bl[c];
  const float* ub = u + (long long)b * npix;
  float* hb = h + (long long)bc * npix;
  // four elements per thread and round (coalesced: the four are blockDim apart), loads before stores
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < npix; i0 += 4 * step) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = i0 + k * step < npix ? ub[i0 + k * step] : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k * step < npix) hb[i0 + k * step] = w0 * v[k] + off;
  }
}

// Second contraction of the truncated transform, per image: out[p][m] = sum_i S[p][i] T[m][i] for
// p, m < M <= 32, i < n (S: the M x n mode matrix S_M; T: the first contraction's [m][i] rows), rounded
// to bf16 when `round`. One CTA of 64 threads per image: both operands' rows in shared memory with the
// odd stride n (distinct banks for the 8 rows a warp reads at one i), each thread a 4 x 4 block of
// outputs (p = tp + 8a, m = tm + 8b) accumulated in FP32 over i in order.
__global__ void __launch_bounds__(64) modes_pm_kernel(const float* __restrict__ S, const float* __restrict__ T,
                                                      float* __restrict__ out, int n, int M, int round) {
  extern __shared__ __align__(16) float sm[];
  float* Ss = sm;
  float* Ts = sm + (size_t)M * n;
  const int img = blockIdx.x, tid = threadIdx.x;
  const float* Ti = T + (size_t)img * M * n;
  // both operands as asynchronous 16-byte copies, all in flight at once (M n is a multiple of 4 and
  // both sources 16-byte aligned when M n is; otherwise element copies)
  const int cnt = M * n;
  if ((cnt & 3) == 0 && ((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(Ti)) & 15) == 0) {
    for (int e = 4 * tid; e < cnt; e += 4 * 64) {
      cp_async16(Ss + e, S + e);
      cp_async16(Ts + e, Ti + e);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else {
    for (int e = tid; e < cnt; e += 64) {
      Ss[e] = S[e];
      Ts[e] = Ti[e];
    }
  }
  __syncthreads();
  const int tp = tid & 7, tm = tid >> 3;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  int pr[4], mr[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    pr[a] = min(tp + 8 * a, M - 1) * n;   // clamped rows: computed, not stored
    mr[a] = min(tm + 8 * a, M - 1) * n;
  }
  for (int i = 0; i < n; ++i) {
    float sv[4], tv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      sv[a] = Ss[pr[a] + i];
      tv[a] = Ts[mr[a] + i];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(sv[a], tv[b], acc[a][b]);
  }
  float* o = out + (size_t)img * M * M;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int pp = tp + 8 * a, mm = tm + 8 * b;
      if (pp < M && mm < M) o[pp * M + mm] = round ? bf16_round(acc[a][b]) : acc[a][b];
    }
}

// First contraction of the inverse truncated transform, per image: T[m][j] = sum_q Y[m][q] S[q][j] for
// m < M <= 32, j < n (Y: the M x M modes; S: S_M). One CTA per image, one output column j per thread
// (coalesced loads of S and stores of T), Y in shared memory read as broadcasts, FP32 accumulation
// over q in order.
__global__ void __launch_bounds__(256, 2) modes_to_rows_kernel(const float* __restrict__ Y, const float* __restrict__ S,
                                                               float* __restrict__ T, int n, int M) {
  __shared__ float Ys[32 * 32];
  const int img = blockIdx.x;
  const float* Yi = Y + (size_t)img * M * M;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) Ys[e] = Yi[e];
  __syncthreads();
  float* Ti = T + (size_t)img * M * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    // the thread's column of S_M in blocks of 8 values, the next block's loads in flight while the current
    // one is used
    float acc[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) acc[m] = 0.f;
    float sv[8], sn[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) sv[k] = k < M ? S[(size_t)k * n + j] : 0.f;
    for (int q0 = 0; q0 < M; q0 += 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int q = q0 + 8 + k;
        sn[k] = q < M ? S[(size_t)q * n + j] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (q0 + k < M) {
#pragma unroll
          for (int m = 0; m < 32; ++m)
            if (m < M) acc[m] = fmaf(Ys[m * M + q0 + k], sv[k], acc[m]);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sv[k] = sn[k];
    }
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < M) Ti[(size_t)m * n + j] = acc[m];
  }
}

// Projection onto the increment: out[b][i] = u[b][i] + bq + sum_c Wq[c] h[b][c][i] (FP32, channels in
// order); grid (pixel blocks, B).
__global__ void __launch_bounds__(256) project_kernel(const float* __restrict__ u, const float* __restrict__ h,
                                                      const float* __restrict__ Wq, const float* __restrict__ bq,
                                                      float* __restrict__ out, int C, long long npix) {
  const int b = blockIdx.y;
  const float* hb = h + (size_t)b * C * npix;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int c = 0; c < C; ++c) acc = fmaf(Wq[c], hb[(size_t)c * npix + i], acc);
    out[(size_t)b * npix + i] = acc + (u[(size_t)b * npix + i] + bq[0]);
  }
}

// dz = dh * gelu'(z)
__global__ void gelu_backward_kernel(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                                     long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dz[e] = dh[e] * gelu_grad(z[e]);
}

// du = 2 (u_hat - target) / count; per-block partial sums of (u_hat - target)^2 in FP64
__global__ void __launch_bounds__(256) mse_grad_kernel(const float* __restrict__ uh, const float* __restrict__ tg,
                                                       float* __restrict__ du, long long n, double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  const float scale = 2.f / (float)n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float d = uh[e] - tg[e];
    du[e] = scale * d;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// part[(bc) * gridDim.x + blk] = partial sums over pixels of X[bc][i] * (y ? y[b][i] : 1), for
// bc = b * C + c = blockIdx.y
__global__ void __launch_bounds__(256) chan_dot_kernel(const float* __restrict__ X, const float* __restrict__ y,
                                                       int C, long long npix, float* __restrict__ part) {
  __shared__ float sh[256];
  const int bc = blockIdx.y, b = bc / C;
  const float* x = X + (long long)bc * npix;
  const float* yy = y ? y + (long long)b * npix : nullptr;
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x)
    s += yy ? x[i] * yy[i] : x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)bc * gridDim.x + blockIdx.x] = sh[0];
}

// out[c * stride] (+)= sum_b w[b] sum_k part[(b * C + c) * nblk + k]   (w = NULL: weights 1)
__global__ void chan_combine_kernel(const float* __restrict__ part, int nblk, const float* __restrict__ w, int B, int C,
                                    float* __restrict__ out, int stride, int accumulate) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) {
    float t = 0.f;
    for (int k = 0; k < nblk; ++k) t += part[((long long)b * C + c) * nblk + k];
    s += (w ? w[b] : 1.f) * t;
  }
  out[(long long)c * stride] = accumulate ? out[(long long)c * stride] + s : s;
}

// out[x] = sum_b in[b * X + x] (+ out[x] when accumulate)
__global__ void reduce_batch_kernel(const float* __restrict__ in, float* __restrict__ out, int B, long long X,
                                    int accumulate) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < X; x += (long long)gridDim.x * blockDim.x) {
    float s = accumulate ? out[x] : 0.f;
    for (int b = 0; b < B; ++b) s += in[(long long)b * X + x];
    out[x] = s;
  }
}

// Adam with bias correction (c1 = 1 - b1^t, c2 = 1 - b2^t)
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gr = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// Parareal update V = Gn + F - Go (V = F where Gn is NULL: a window from a start that is already the
// fine solution), and per-problem squared norms of V and of V - U (FP64 partials, one block row per
// problem: blockIdx.y = problem)
__global__ void __launch_bounds__(256) parareal_update_kernel(const float* __restrict__ Gn, const float* __restrict__ F,
                                                              const float* __restrict__ Go, const float* __restrict__ U,
                                                              float* __restrict__ V, long long npix,
                                                              double* __restrict__ part /* [B][gridDim.x][2] */) {
  __shared__ double s0[256], s1[256];
  const long long base = (long long)blockIdx.y * npix;
  double a = 0.0, d = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
    const float v = Gn ? Gn[base + i] + F[base + i] - Go[base + i] : F[base + i];
    V[base + i] = v;
    const float e = v - U[base + i];
    a += (double)v * v;
    d += (double)e * e;
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = d;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      s0[threadIdx.x] += s0[threadIdx.x + k];
      s1[threadIdx.x] += s1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 0] = s0[0];
    part[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = s1[0];
  }
}

}  // namespace sno
}  // namespace etd
