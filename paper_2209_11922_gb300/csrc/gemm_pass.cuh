// gemm_pass.cuh - tensor-core transform pass: the sine transform of Section 4 along one axis as a
// dense contraction on the tcgen05 tensor cores, with the pointwise work of the step fused into
// the epilogue and the result written transposed.
//
// A field is a pitched array of R rows of K = N_a values, the contracted axis a contiguous (index 0
// of every axis is the boundary, value 0). One pass computes C = X S_a, C[r][k] = sum_j X[r][j]
// S_a[j][k] with S_a[j][k] = sqrt(2/N_a) sin(j k pi / N_a) (j, k < N_a; row and column 0 vanish, so
// boundary values stay 0), and writes epi(C[r][k]) to out[k * R + r]. Periodic plans contract with
// the orthonormal Hartley matrix N_a^{-1/2} cas(2 pi j k / N_a) instead (every index is a node), which
// is also symmetric and its own inverse; the pass itself does not depend on the matrix. Writing the transpose rotates
// the axes: [z][y][x] -> [x][z][y] -> [y][x][z] -> [z][y][x] (2D: [y][x] -> [x][y] -> [y][x]), so
// every pass contracts a contiguous axis and d passes return to the starting layout.
//
// Operand formats (route):
//   TF32      X fp32 as stored, S rounded to TF32 once on the host; kind::tf32.
//   BF16x3    X = X_hi + X_lo, S = S_hi + S_lo with bf16 parts (X split in shared memory as each
//             tile arrives), C = X_hi S_hi + X_hi S_lo + X_lo S_hi; kind::f16 with BF16 operands.
// Accumulation is FP32 in tensor memory for both.
//
// CTA: 128 rows x BN columns of C, 320 threads. Warp 0 issues the TMA loads, warp 1 owns the
// tensor memory and issues the MMAs, warps 2-9 split the operand tile (BF16x3) and run the epilogue
// (warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. rows r0 + 32 (w % 4) + lane; warps 2-5 take the
// first BN/2 columns, warps 6-9 the rest).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "etd_coeffs.cuh"
#include "umma.cuh"

namespace etd {

enum GemmEpi : int { GE_PLAIN = 0, GE_REACT = 1, GE_RK1 = 2, GE_S1 = 3, GE_S2 = 4 };
enum GemmRoute : int { GR_TF32 = 0, GR_BF16X3 = 1 };

struct GemmArgs {
  int op;            // GemmEpi
  int R;             // rows of the input field
  int K;             // length of the contracted axis (multiple of 32)
  int row_split;     // 3D spectral passes: r = y * row_split + x; 0: r = x (2D)
  const float* in1;  // V (RK1, S1) or P (S2), in the output layout
  float* out0;
  float* out1;       // P (S1)
  // per-mode tables (zeta = tau D mu_i, exp(-zeta), exp(-c2 zeta)) of the row axes and the column
  // (contracted) axis of the spectral passes
  const float* zx; const float* ex; const float* cx;
  const float* zy; const float* ey; const float* cy;
  const float* zk; const float* ek; const float* ck;
  float tau, c2, flin, fcub, flog;   // f(u) = flin u + fcub u^3 + flog artanh u
  int* err;          // set to 1 by a CTA whose wait ran out
  int stall;         // test of the failure path: the accumulator-ready signal is withheld
};

struct GemmParams {
  CUtensorMap ta;    // X: fp32 [R][K], box {32, 128}, 128-byte swizzle
  CUtensorMap tb0;   // TF32: S fp32 [K][K] box {32, BN}, 128-byte swizzle; BF16x3: S_hi bf16, box {32, BN}, 64-byte swizzle
  CUtensorMap tb1;   // BF16x3: S_lo (as tb0); TF32: unused
  GemmArgs g;
};

template <int BN> struct GemmShape {
  static constexpr int BM = 128, BK = 32;                         // BK: K per stage (128 B of fp32)
  static constexpr uint32_t A_BYTES = BM * BK * 4;                // 16 KB
  static constexpr uint32_t B_BYTES = BN * BK * 4;                // fp32 tile, or two bf16 tiles
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  // about 96 KB of stages: two CTAs per SM (2 x BN <= 512 tensor-memory columns)
  static constexpr int NSTAGE = (98304 / STAGE) < 2 ? 2 : ((98304 / STAGE) > 6 ? 6 : (98304 / STAGE));
  static constexpr uint32_t BAR_BYTES = 256;
  static constexpr uint32_t TAB_BYTES = 3 * BN * 4;                 // per-column mode tables
  static constexpr size_t SMEM = 1024 + (size_t)NSTAGE * STAGE + BAR_BYTES + TAB_BYTES;   // + alignment slack
  static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "BN");
  static_assert((4 * NSTAGE + 1) * 8 + 8 <= BAR_BYTES, "barrier area");
};

// fp32 -> (hi, lo) bf16 pairs of 8 values, packed 2 per 32-bit word
__device__ __forceinline__ void split8(const float4& a, const float4& b, uint4& hi, uint4& lo) {
  const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]), h1 = __float2bfloat16_rn(v[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
    h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Pointwise epilogue of columns [cb, ce) of the 128 x BN accumulator tile for row r: C[r][k] from
// tensor memory, epi applied, written to out[k * R + r] (consecutive lanes -> consecutive
// addresses). tabs holds zeta, exp(-zeta), exp(-c2 zeta) of the tile's BN columns.
template <int BN>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs& g, uint32_t trow, int r, int n0, int cb, int ce,
                                              const float* __restrict__ tabs) {
  const bool row_ok = r < g.R;
  const int op = g.op;
  const bool spectral = op == GE_RK1 || op == GE_S1 || op == GE_S2;
  float zr = 0.f, er = 1.f, cr = 1.f;   // row part of zeta, exp(-zeta), exp(-c2 zeta)
  if (spectral && row_ok) {
    int x = r, y = 0;
    if (g.row_split > 0) {
      y = r / g.row_split;
      x = r - y * g.row_split;
    }
    zr = g.zx[x];
    er = g.ex[x];
    cr = g.cx[x];
    if (g.row_split > 0) {
      zr += g.zy[y];
      er *= g.ey[y];
      cr *= g.cy[y];
    }
  }
  const float tau = g.tau, c2 = g.c2, flin = g.flin, fcub = g.fcub, inv_c2 = 1.f / g.c2;
  const int R = g.R;   // fields hold < 2^31 values: per-column offsets j * R in 32 bits
  // second input of the spectral passes, one chunk ahead: the loads of chunk c + 16 are in flight
  // while chunk c is computed
  float wn[16];
  auto load_w = [&](int c) {
    const int kb = n0 + c;
    const int nv = g.K - kb < 16 ? g.K - kb : 16;
    const float* i1 = g.in1 + (size_t)kb * (size_t)R + r;
#pragma unroll
    for (int j = 0; j < 16; ++j) wn[j] = j < nv ? i1[j * R] : 0.f;
  };
  if (spectral && row_ok && cb < ce) load_w(cb);
  for (int c0 = cb; c0 < ce; c0 += 16) {
    float v[16];
    umma::tmem_ld16(trow + (uint32_t)c0, v);   // warp-collective: every lane takes part
    if (!row_ok) continue;
    const int kb = n0 + c0;
    const int nv = g.K - kb < 16 ? g.K - kb : 16;   // valid columns of this chunk
    float* o0 = g.out0 + (size_t)kb * (size_t)R + r;
    if (op == GE_PLAIN) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nv) o0[j * R] = v[j];
      continue;
    }
    if (op == GE_REACT) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nv) {
          float fr = v[j] * (flin + fcub * v[j] * v[j]);
          if (g.flog != 0.f) fr += g.flog * atanhf(v[j]);
          o0[j * R] = fr;
        }
      continue;
    }
    // spectral combination
    float w[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) w[j] = wn[j];
    if (c0 + 16 < ce) load_w(c0 + 16);
    const float* tz = tabs + c0;
    const float* te = tabs + BN + c0;
    const float* tc = tabs + 2 * BN + c0;
    float* o1 = op == GE_S1 ? g.out1 + (size_t)kb * (size_t)R + r : nullptr;
    // phi_k(-zeta) in closed form for zeta >= 1: one reciprocal per mode serves phi_1, phi_2 and
    // the c2 stage. The modes grow along the column axis, so the smallest zeta of this chunk is at
    // its first column: a warp none of whose rows needs the series there (zeta < 1, or
    // c2 zeta < 1 in the first stage) takes the closed-form-only loop for all 16 columns; warps
    // in the low-mode corner of the spectrum take the general loop. Rows come in whole warps (R is
    // a multiple of 32), so every lane of a warp reaches the vote.
    const unsigned act = __activemask();
    const float zcut = op == GE_S1 ? inv_c2 : 1.f;
    if (!__any_sync(act, zr + tz[0] < zcut)) {
      const float tau_c2 = tau * inv_c2;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float zeta = zr + tz[j], E = er * te[j];
        const float rz = rcp_approx(zeta);   // 1 ulp: far below the route's TF32 / bf16 error
        const float p1 = (1.f - E) * rz;
        float out;
        if (op == GE_RK1) {
          out = E * w[j] + tau * p1 * v[j];
        } else {
          const float p2 = (1.f - p1) * rz;
          if (op == GE_S2) {
            out = w[j] + tau_c2 * p2 * v[j];
          } else {
            const float Ec = cr * tc[j];
            out = Ec * w[j] + tau * (1.f - Ec) * rz * v[j];   // c2 tau phi1(-c2 zeta), c2 zeta >= 1
            if (j < nv) o1[j * R] = E * w[j] + tau * (p1 - p2 * inv_c2) * v[j];
          }
        }
        if (j < nv) o0[j * R] = out;
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float zeta = zr + tz[j], E = er * te[j];
      const float rz = rcp_approx(fmaxf(zeta, 1.f));
      float p1 = (1.f - E) * rz, p2 = (1.f - p1) * rz;
      const bool small = zeta < 1.f;
      if (__any_sync(act, small)) {
        const float s2 = phi2_series<float>(small ? -zeta : 0.f);
        p2 = small ? s2 : p2;
        p1 = small ? 1.f - zeta * s2 : p1;
      }
      float out;
      if (op == GE_RK1) {
        out = E * w[j] + tau * p1 * v[j];
      } else if (op == GE_S2) {
        out = w[j] + (tau * inv_c2) * p2 * v[j];
      } else {
        const float Ec = cr * tc[j], zc = c2 * zeta;
        // c2 tau phi1(-c2 zeta) = tau (1 - Ec) / zeta for c2 zeta >= 1
        float t1 = tau * (1.f - Ec) * rz;
        if (__any_sync(act, zc < 1.f)) {
          const bool sm = zc < 1.f;
          const float s2c = phi2_series<float>(sm ? -zc : 0.f);
          t1 = sm ? c2 * tau * (1.f - zc * s2c) : t1;
        }
        out = Ec * w[j] + t1 * v[j];
        if (j < nv) o1[j * R] = E * w[j] + tau * (p1 - p2 * inv_c2) * v[j];
      }
      if (j < nv) o0[j * R] = out;
    }
  }
}

constexpr int kGemmThreads = 320;   // warp 0 TMA, warp 1 MMA, warps 2-9 split + epilogue

template <int BN, int ROUTE>
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_pass_kernel(const __grid_constant__ GemmParams prm) {
  using G = GemmShape<BN>;
  constexpr int BM = G::BM, BK = G::BK, NS = G::NSTAGE;
  const GemmArgs& g = prm.g;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)NS * G::STAGE);   // TMA -> consumers
  uint64_t* empty = full + NS;                                                // MMA done with a stage
  uint64_t* conv = empty + NS;                                                // BF16x3: tile split
  uint64_t* accf = conv + NS;                                                 // accumulator complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  float* tabs = reinterpret_cast<float*>(sm + (size_t)NS * G::STAGE + G::BAR_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = (g.R + BM - 1) / BM;
  const int r0 = (int)(blockIdx.x % m_tiles) * BM, n0 = (int)(blockIdx.x / m_tiles) * BN;
  const int nk = g.K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
      umma::mbar_init(&conv[s], 8);
    }
    umma::mbar_init(accf, 1);
    *abort_flag = 0;
    umma::mbar_fence_init();
  }
  if (warp == 1) umma::tmem_alloc(tslot, BN);
  if (warp >= 2 && (g.op == GE_RK1 || g.op == GE_S1 || g.op == GE_S2)) {
    // per-column tables of this tile (constant tables: read before the dependency wait)
    for (int i = threadIdx.x - 64; i < BN; i += kGemmThreads - 64) {
      const int k = n0 + i < g.K ? n0 + i : g.K - 1;
      tabs[i] = g.zk[k];
      tabs[BN + i] = g.ek[k];
      tabs[2 * BN + i] = g.ck[k];
    }
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = *tslot;
  griddep_wait();   // the field is written by the previous pass

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % NS;
        const uint32_t ph = (uint32_t)(i / NS) & 1u;
        if (i >= NS && !umma::mbar_wait(&empty[s], ph ^ 1u, abort_flag, g.err)) break;
        unsigned char* st = sm + (size_t)s * G::STAGE;
        umma::mbar_arrive_expect_tx(&full[s], G::STAGE);
        umma::tma_load_2d(st, &prm.ta, &full[s], i * BK, r0);
        umma::tma_load_2d(st + G::A_BYTES, &prm.tb0, &full[s], i * BK, n0);
        if (ROUTE == GR_BF16X3) umma::tma_load_2d(st + G::A_BYTES + G::B_BYTES / 2, &prm.tb1, &full[s], i * BK, n0);
        issued = i + 1;
      }
      if (*abort_flag)   // copies already issued land before the shared memory is released
        for (int i = issued > NS ? issued - NS : 0; i < issued; ++i)
          umma::mbar_drain(&full[i % NS], (uint32_t)(i / NS) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      constexpr uint32_t IDESC = umma::instr_desc(ROUTE == GR_TF32 ? 2u : 1u, BM, BN);
      for (int i = 0; i < nk; ++i) {
        const int s = i % NS;
        const uint32_t ph = (uint32_t)(i / NS) & 1u;
        if (!umma::mbar_wait(ROUTE == GR_TF32 ? &full[s] : &conv[s], ph, abort_flag, g.err)) break;
        umma::tc_fence_after();
        const uint32_t a = umma::smem_addr(sm + (size_t)s * G::STAGE);
        const uint32_t b = a + G::A_BYTES;
        if (ROUTE == GR_TF32) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)   // 8 TF32 values = 32 bytes of K per instruction
            umma::mma_tf32(tmem, umma::smem_desc(a + 32 * kk, 1024, umma::kSwizzle128),
                           umma::smem_desc(b + 32 * kk, 1024, umma::kSwizzle128), IDESC, (i | kk) != 0);
        } else {
          const uint32_t alo = a + 8192, blo = b + G::B_BYTES / 2;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {   // 16 BF16 values = 32 bytes of K per instruction
            const uint64_t ah = umma::smem_desc(a + 32 * kk, 512, umma::kSwizzle64);
            const uint64_t al = umma::smem_desc(alo + 32 * kk, 512, umma::kSwizzle64);
            const uint64_t bh = umma::smem_desc(b + 32 * kk, 512, umma::kSwizzle64);
            const uint64_t bl = umma::smem_desc(blo + 32 * kk, 512, umma::kSwizzle64);
            umma::mma_bf16(tmem, al, bh, IDESC, (i | kk) != 0);   // small products first
            umma::mma_bf16(tmem, ah, bl, IDESC, 1);
            umma::mma_bf16(tmem, ah, bh, IDESC, 1);
          }
        }
        umma::mma_commit(&empty[s]);
      }
      if (!g.stall) umma::mma_commit(accf);
      if (*abort_flag) umma::mbar_drain(accf, 0);   // MMAs in flight finish before TMEM is freed
    }
  } else {
    const int e = threadIdx.x - 64;      // 0..255
    const int half = e >> 7;             // column half (epilogue) / chunk half (split)
    const int rl = 32 * (warp & 3) + lane;   // row within the tile = TMEM lane (warp w reads lanes 32 (w % 4) ..)
    if (ROUTE == GR_BF16X3) {
      // Split the fp32 tile in place: row rl (128 B, 128-byte swizzle) -> hi row at rl * 64 and lo
      // row at 8192 + rl * 64 (64-byte swizzle); thread half h converts fp32 chunks 4h..4h+3. Rows
      // of other threads overlap, so every converter thread reads before any writes (one named
      // barrier per stage, always executed).
      for (int i = 0; i < nk; ++i) {
        const int s = i % NS;
        const uint32_t ph = (uint32_t)(i / NS) & 1u;
        const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&full[s], ph, abort_flag, g.err));
        unsigned char* st = sm + (size_t)s * G::STAGE;
        float4 v[4];
        if (ok) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            v[c] = *reinterpret_cast<const float4*>(st + rl * 128 + (((4 * half + c) ^ (rl & 7)) << 4));
        }
        __syncwarp();
        umma::named_barrier(1, kGemmThreads - 64);
        if (ok) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint4 hi, lo;
            split8(v[2 * c], v[2 * c + 1], hi, lo);
            const int pos = ((2 * half + c) ^ ((rl >> 1) & 3)) << 4;
            *reinterpret_cast<uint4*>(st + rl * 64 + pos) = hi;
            *reinterpret_cast<uint4*>(st + 8192 + rl * 64 + pos) = lo;
          }
          umma::fence_proxy_async();
        }
        __syncwarp();
        if (ok && lane == 0) umma::mbar_arrive(&conv[s]);
      }
    }
    const bool got = __all_sync(0xffffffffu, umma::mbar_wait(accf, 0, abort_flag, g.err));
    umma::tc_fence_after();
    griddep_launch_dependents();
    if (got)
      gemm_epilogue<BN>(g, tmem + ((uint32_t)(32 * (warp & 3)) << 16), r0 + rl, n0, half * (BN / 2),
                        (half + 1) * (BN / 2), tabs);
  }
  __syncwarp();
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tmem, BN);
  }
}

// Host-side handle of one instantiation.
struct GemmKernelInfo {
  const void* fn;
  int bn, route;
  size_t smem;
  int threads;
};
template <int BN, int ROUTE> GemmKernelInfo gemm_kernel_info() {
  return GemmKernelInfo{reinterpret_cast<const void*>(&gemm_pass_kernel<BN, ROUTE>), BN, ROUTE, GemmShape<BN>::SMEM,
                        kGemmThreads};
}

}  // namespace etd
