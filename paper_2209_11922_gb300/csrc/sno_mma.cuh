// sno_mma.cuh - the large contractions of the spectral neural operator's forward pass on the
// tcgen05 tensor cores, BF16 operands and FP32 accumulation (kind::f16):
//   T1  the truncated sine transform along x, T[img][m][i] = sum_j bf(X[img][i][j]) bf(S_M[m][j]),
//   F2  the inverse truncated transform along y, out[img][i][j] (+)= sum_m bf(S_M[m][i]) bf(T[img][m][j]),
//   PW  the pointwise channel mix of a layer, z[b][o][i] = sum_c bf(Wp[o][c]) bf(h[b][c][i]) + z + bp[o],
//       h'[b][o][i] = gelu(z) (ME_PW_GELU stores z too, for the gradient; ME_PW_GELU_ONLY only h'),
// each as D[r][c] = sum_k A[r][k] B[c][k] over tiles of 128 rows r, with every output column c of the
// contraction in one tile (c < NCOL <= 256) and the whole K (<= 256) resident.
//
// A CTA (8 warps) stages the constant operand B once, then loops over row tiles: all threads convert
// the tile's A rows from FP32 global memory to BF16 in shared memory (K-major, 64-byte rows, swizzled
// as the tensor core reads them: 16-byte chunk q of row r at chunk position q ^ ((r / 2) % 4), 8-row
// atoms of 512 bytes, one 128 x 32 block per 32 values of K), one thread issues the MMAs (K = 16 per
// instruction) and commits them to an mbarrier, and each warp reads 32 rows and half the columns of
// the accumulator from tensor memory for the fused epilogue. Waits are limited in time (umma::mbar_wait); a CTA that
// runs out sets the error word and stops.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sno_kernels.cuh"
#include "umma.cuh"

namespace etd {
namespace sno {

enum MmaEpi : int { ME_STORE = 0, ME_ACCUM = 1, ME_PW_GELU = 2, ME_PW_GELU_ONLY = 3 };

struct MmaArgs {
  int tiles_per_img, imgs;       // tile t: image t / tiles_per_img, rows r0 = 128 (t % tiles_per_img)
  int rows;                      // valid rows per image
  int kvalid, kpad;              // K used (<= kpad), kpad a multiple of 32, <= 256
  int ncol;                      // valid output columns (<= NCOL)
  const float* A;                // A[img][r][k] = A[img a_is + r a_rs + k a_ks]
  long long a_rs, a_ks, a_is;
  const float* B;                // B[c][k] = B[c b_cs + k b_ks], shared by every tile
  long long b_cs, b_ks;
  float* C;                      // output (img, r, c) at C[img c_is + r c_rs + c c_cs]
  long long c_rs, c_cs, c_is;
  float beta;                    // ME_ACCUM, ME_PW_GELU: C = D + beta C (+ bias)
  const float* bias;             // ME_PW_GELU: [ncol]
  float* C2;                     // ME_PW_GELU: gelu(C), C's layout
  int* err;                      // set when a wait runs out
};

// bytes of shared memory: A blocks, B blocks, barrier + TMEM slot + abort flag, 1 KB alignment slack
__host__ __device__ constexpr size_t mma_smem_bytes(int ncol, int kpad) {
  return 1024 + (size_t)(kpad / 32) * (128 + ncol) * 64 + 64;
}

// fp32 x 8 -> bf16 x 8 (round to nearest even), packed two per 32-bit word
__device__ __forceinline__ uint4 pack_bf16x8(const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i])) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i + 1])) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Stages R x kpad values M[r][k] = src[r rs + k ks] (0 outside r < rvalid, k < kvalid) as bf16 into
// the swizzled K-major blocks at dst (block kc of R x 64 bytes holds k = 32 kc .. 32 kc + 31). An item
// is 8 consecutive k of one row (one 16-byte chunk). K-contiguous sources (ks = 1): eight consecutive
// items fill two adjacent rows of one block, so a warp's stores cover 512 contiguous bytes (no bank
// conflicts) and its loads read 8 rows of 128 bytes. Other sources: consecutive items take consecutive
// rows (coalesced loads along r). Each thread takes four items per round and issues all their loads
// before converting any, to keep enough loads in flight.
__device__ __forceinline__ void stage_bf16(unsigned char* dst, int R, const float* __restrict__ src, long long rs,
                                           long long ks, int rvalid, int kvalid, int kpad, int tid, int nt) {
  constexpr int U = 4;
  const int q8 = kpad / 8;   // items per row
  const int total = R * q8;
  const bool kfast = ks == 1;
  for (int base = tid; base < total; base += U * nt) {
    float v[U][8];
    int off[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = base + u * nt;
      int r, q;
      if (kfast) {
        const int kc = it / (4 * R), rem = it - kc * 4 * R;
        r = rem >> 2;
        q = 4 * kc + (rem & 3);
      } else {
        q = it / R;
        r = it - q * R;
      }
      const bool ok = it < total;
      off[u] = ok ? (q >> 2) * R * 64 + r * 64 + (((q & 3) ^ ((r >> 1) & 3)) << 4) : -1;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = 8 * q + e;
        v[u][e] = (ok && r < rvalid && k < kvalid) ? src[(long long)r * rs + (long long)k * ks] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (off[u] >= 0) *reinterpret_cast<uint4*>(dst + off[u]) = pack_bf16x8(v[u]);
  }
}

constexpr int kMmaThreads = 256;   // 8 warps: warps w and w + 4 read accumulator lanes 32 (w mod 4) ..

// Narrow tiles (NCOL <= 64: the pointwise mix and the truncated transform) are held to 64 registers so that
// four CTAs (32 warps) share an SM and keep their loads in flight; wider tiles are limited by their tensor
// memory to two CTAs per SM anyway.
template <int NCOL, int EPI>
__global__ void __launch_bounds__(kMmaThreads, NCOL <= 64 ? 4 : 1) sno_mma_kernel(const MmaArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sA =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int nkc = g.kpad / 32;
  unsigned char* sB = sA + (size_t)nkc * 128 * 64;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + (size_t)nkc * NCOL * 64);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    umma::mbar_init(bar, 1);
    *abort_flag = 0;
    umma::mbar_fence_init();
  }
  if (warp == 0) umma::tmem_alloc(tslot, NCOL < 32 ? 32 : NCOL);
  stage_bf16(sB, NCOL, g.B, g.b_cs, g.b_ks, g.ncol, g.kvalid, g.kpad, tid, kMmaThreads);
  umma::fence_proxy_async();
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t IDESC = umma::instr_desc(1u, 128, NCOL);   // BF16 x BF16 -> FP32, M = 128
  constexpr int CW = NCOL / 2;                                   // accumulator columns per warp
  const int lg = warp & 3, half = warp >> 2;
  const int ntiles = g.tiles_per_img * g.imgs;
  uint32_t phase = 0;
  bool ok = true;
  for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int img = t / g.tiles_per_img, r0 = (t % g.tiles_per_img) * 128;
    stage_bf16(sA, 128, g.A + (long long)img * g.a_is + (long long)r0 * g.a_rs, g.a_rs, g.a_ks, g.rows - r0,
               g.kvalid, g.kpad, tid, kMmaThreads);
    umma::fence_proxy_async();
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    if (tid == 0) {
      for (int kc = 0; kc < nkc; ++kc)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint64_t da = umma::smem_desc(umma::smem_addr(sA + (size_t)kc * 128 * 64 + 32 * kk), 512, umma::kSwizzle64);
          const uint64_t db = umma::smem_desc(umma::smem_addr(sB + (size_t)kc * NCOL * 64 + 32 * kk), 512, umma::kSwizzle64);
          umma::mma_bf16(tmem, da, db, IDESC, (kc | kk) != 0);
        }
      umma::mma_commit(bar);
    }
    // epilogue: warp w holds rows r0 + 32 (w mod 4) + lane (accumulator lanes 32 (w mod 4) ..) and
    // columns [CW (w / 4), CW (w / 4 + 1)); the values the epilogue adds to are loaded before the wait
    const int r = r0 + 32 * lg + lane;
    const bool rv = r < g.rows;
    float* C = g.C + (long long)img * g.c_is + (long long)r * g.c_rs;
    float cpre[CW < 16 ? CW : 16];
    if constexpr (EPI != ME_STORE && CW == 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = half * CW + i;
        cpre[i] = (rv && c < g.ncol) ? C[(long long)c * g.c_cs] : 0.f;
      }
    }
    ok = __all_sync(0xffffffffu, umma::mbar_wait(bar, phase, abort_flag, g.err));
    phase ^= 1u;
    umma::tc_fence_after();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
#pragma unroll 1
    for (int c0 = half * CW; c0 < (half + 1) * CW; c0 += 16) {
      float cv[16];
      if constexpr (EPI != ME_STORE) {
        if constexpr (CW == 16) {
#pragma unroll
          for (int i = 0; i < 16; ++i) cv[i] = cpre[i];
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            cv[i] = (rv && c < g.ncol) ? C[(long long)c * g.c_cs] : 0.f;
          }
        }
      }
      float v[16];
      umma::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)c0, v);
      if (!rv) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = c0 + i;
        if (c >= g.ncol) break;
        float* p = C + (long long)c * g.c_cs;
        if constexpr (EPI == ME_STORE) {
          *p = v[i];
        } else if constexpr (EPI == ME_ACCUM) {
          *p = v[i] + g.beta * cv[i];
        } else {
          const float z = v[i] + g.beta * cv[i] + g.bias[c];
          if constexpr (EPI == ME_PW_GELU) *p = z;
          g.C2[(long long)img * g.c_is + (long long)r * g.c_rs + (long long)c * g.c_cs] = gelu(z);
        }
      }
    }
    umma::tc_fence_before();
    __syncthreads();   // the accumulator and the A blocks are free for the next tile
    umma::tc_fence_after();
  }
  if (tid == 0 && *abort_flag) umma::mbar_drain(bar, phase);   // MMAs in flight finish before TMEM is freed
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tmem, NCOL < 32 ? 32 : NCOL);
  }
}

}  // namespace sno
}  // namespace etd
