// split_pass.cuh - FP32 axis passes of the fast EIFE solve (Section 4) for axes of N = 1024 intervals,
// built on the split-radix DST-I of split_dst.cuh. One kernel per pass kind (template OP, the PassOp
// values of pass_kernel.cuh), same arguments (PassArgs<float>) and the same field layouts as pass_kernel:
//   ENTRY / EXIT / REACT        x axis (contiguous rows): tiles of P = 2 pencil pairs (4 rows), 5 warps
//   TRANSFORM                   any axis
//   S1 / RK1                    last axis (strided): tiles of P pairs of adjacent x columns; the two input
//                               fields are transformed by two warp sets at once (10 warps per 2 pairs)
//   S2                          last axis: one transformed field plus the P field
// Position 0 of every pencil (the boundary node, or sine mode 0) is loaded as an exact zero. Pair packing
// puts two real pencils into one complex transform, so the boundary row or column of the other axis comes
// back from a pass with rounding noise in it (the real part of the transform of a purely imaginary pencil
// vanishes only in exact arithmetic); the gathers read position 0, and noise there would enter every
// sub-transform's zero-frequency term.
// A tile's pairs are grouped two by two; each group takes five warps: A of pair 0 and 1, C of pair 0 and 1,
// B of both (one half-warp each). A transform in place is gather + FFT (registers and per-warp
// scratch), one barrier of the group, scatter, one barrier of the group; the nodal reaction f(u) = flin u + fcub u^3 of REACT is applied
// as the inverse transform writes its nodal values, and the spectral stage combinations of eqs.
// (2.13)/(2.14) run as a pointwise pass over the tile between the forward and the inverse transform.
#pragma once
#include <type_traits>

#include "etd_coeffs.cuh"
#include "pass_kernel.cuh"
#include "split_dst.cuh"

namespace etd {

template <int OP> struct SplitOp {
  static constexpr bool SPECTRAL = OP == OP_S1 || OP == OP_S2 || OP == OP_RK1;
  static constexpr int NB = SPECTRAL ? 2 : 1;                          // tile buffer sets
  static constexpr int NF = (OP == OP_S1 || OP == OP_RK1) ? 2 : 1;     // buffer sets transformed at once
  // threads: P = 2 pairs along x (5 warps), P = 4 along strided axes (10 warps per transformed set)
  static constexpr int MAXT = (OP == OP_ENTRY || OP == OP_EXIT || OP == OP_REACT) ? 160 : NF * 320;
};

// shared memory of a split pass with P pairs per tile and the CTA's warp count
inline size_t split_smem_bytes(int op, int P) {
  const bool spec = op == OP_S1 || op == OP_S2 || op == OP_RK1;
  const int nb = spec ? 2 : 1, nf = (op == OP_S1 || op == OP_RK1) ? 2 : 1;
  const int warps = nf * (P / 2) * 5;
  size_t b = (size_t)SPLIT_TWN * 8 + (size_t)nb * P * SPLIT_LPS * 8 + (size_t)warps * SPLIT_SCR * 8;
  if (spec) b += (3 * (size_t)SPLIT_N + 3 * 2 * (size_t)P) * 4;
  return b;
}

// Stage combination of eqs. (2.13)/(2.14) over the tile, mode by mode: buffer set 0 holds the transformed
// first field (S1, RK1: U~; S2: N2~), set 1 the second (S1, RK1: N0~; S2: P). Writes U2~ (S1), U~+ (RK1,
// S2) into set 0 and P (S1) into set 1. With per-mode tables of the phi-function weights (A.coef, FP32
// values of FP64 phi-functions, [y mode][x mode]) a mode costs two fused multiply-adds per output and
// e^{-z}, e^{-c2 z} are products of the per-axis factors; without them (3D) every coefficient is
// evaluated here in FP32 from zeta = tau D (mu_x + mu_y [+ mu_z]).
template <int OP>
__device__ __forceinline__ void split_epilogue(const PassArgs<float>& A, int P, Cf* bufs, const float* tz,
                                               const float* te, const float* tc, const float* qz, const float* qe,
                                               const float* qc, int x0, int tid, int NT) {
  constexpr int N = SPLIT_N;
  if (A.coef) {
    // A thread's items are it = tid + i NT (p = it % P fastest, so that a warp reads whole table rows);
    // every table load is issued before the first use, so the CTA waits for one L2 latency.
    constexpr int IT = (OP == OP_S2) ? 13 : 7;      // P N / NT = 2 N / (160 NF), rounded up
    constexpr int CH = (OP == OP_S2) ? 13 : 4;      // items whose loads are issued together
    using CT = typename std::conditional<OP == OP_S1, float4, float2>::type;
    const CT* tab = reinterpret_cast<const CT*>(A.coef);
#pragma unroll
    for (int i0 = 0; i0 < IT; i0 += CH) {
      CT cf[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int it = tid + (i0 + i) * NT;
        if (i0 + i < IT && it < P * N) cf[i] = tab[((size_t)(it / P) * A.nx + x0 + 2 * (it % P)) / 2];
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int it = tid + (i0 + i) * NT;
        const int p = it % P, j = it / P;
        if (i0 + i >= IT || it >= P * N || j == 0) continue;
        Cf* b0 = bufs + p * SPLIT_LPS + sslot(j);
        Cf* b1 = bufs + (P + p) * SPLIT_LPS + sslot(j);
        const Cf u = *b0, w = *b1;
        if constexpr (OP == OP_S1) {     // table {c2 tau phi1(-c2 z), tau (phi1 - phi2/c2)(-z)} per mode
          const float Ea = qe[2 * p] * te[j], Eb = qe[2 * p + 1] * te[j];
          const float Ca = qc[2 * p] * tc[j], Cb = qc[2 * p + 1] * tc[j];
          *b0 = Cf{fmaf(Ca, u.x, cf[i].x * w.x), fmaf(Cb, u.y, cf[i].z * w.y)};
          *b1 = Cf{fmaf(Ea, u.x, cf[i].y * w.x), fmaf(Eb, u.y, cf[i].w * w.y)};
        } else if constexpr (OP == OP_RK1) {   // table tau phi1(-z) per mode
          const float Ea = qe[2 * p] * te[j], Eb = qe[2 * p + 1] * te[j];
          *b0 = Cf{fmaf(Ea, u.x, cf[i].x * w.x), fmaf(Eb, u.y, cf[i].y * w.y)};
        } else {                          // S2, table tau phi2(-z) / c2 per mode; b0 = N2~, b1 = P
          *b0 = Cf{fmaf(cf[i].x, u.x, w.x), fmaf(cf[i].y, u.y, w.y)};
        }
      }
    }
    return;
  }
  const float tau = A.tau, c2 = A.c2, inv_c2 = 1.f / A.c2;
  for (int it = tid; it < P * N; it += NT) {
    const int p = it / N, j = it % N;
    if (j == 0) continue;
    Cf* b0 = bufs + p * SPLIT_LPS + sslot(j);
    Cf* b1 = bufs + (P + p) * SPLIT_LPS + sslot(j);
    const Cf u = *b0, w = *b1;
    const float uv[2] = {u.x, u.y}, wv[2] = {w.x, w.y};
    float o0[2], o1[2];
    const unsigned act = __activemask();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float zeta = qz[2 * p + s] + tz[j], E = qe[2 * p + s] * te[j];
      float p1, p2, rz;
      stage_phi12<float>(zeta, E, act, p1, p2, rz);
      if constexpr (OP == OP_RK1) {
        o0[s] = E * uv[s] + tau * p1 * wv[s];
      } else if constexpr (OP == OP_S1) {
        const float Ec = qc[2 * p + s] * tc[j];
        const float t1 = tau * stage_phi1c<float>(zeta, Ec, c2, rz, act);   // c2 tau phi1(-c2 zeta)
        o0[s] = Ec * uv[s] + t1 * wv[s];                          // U2~
        o1[s] = E * uv[s] + tau * (p1 - p2 * inv_c2) * wv[s];      // P
      } else {   // S2: b0 = N2~, b1 = P
        o0[s] = wv[s] + (tau * inv_c2) * p2 * uv[s];
      }
    }
    *b0 = Cf{o0[0], o0[1]};
    if constexpr (OP == OP_S1) *b1 = Cf{o1[0], o1[1]};
  }
}

template <int OP>
__global__ void __launch_bounds__(SplitOp<OP>::MAXT) split_kernel(const PassArgs<float> A) {
  using C = Cf;
  constexpr int N = SPLIT_N;
  constexpr int LPS = SPLIT_LPS;
  constexpr int NB = SplitOp<OP>::NB;
  constexpr int NF = SplitOp<OP>::NF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tab = reinterpret_cast<C*>(smem_raw);
  C* bufs = tab + SPLIT_TWN;
  const int P = A.P;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
  C* scr = bufs + NB * P * LPS;
  float* tz = reinterpret_cast<float*>(scr + (NT / 32) * SPLIT_SCR);   // spectral ops: transformed axis tables
  float* te = tz + N;
  float* tc = te + N;
  float* qz = tc + N;                                                  // per pencil of the tile
  float* qe = qz + 2 * P;
  float* qc = qe + 2 * P;
  const bool contiguous = (A.axis == 0);

  // ---- tile geometry (as pass_kernel)
  int q0 = 0, stride = 0, x0 = 0, o = 0;
  long long base = 0;
  if (contiguous) {
    q0 = blockIdx.x * P;
  } else {
    const int xt = blockIdx.x % A.tiles_x;
    o = blockIdx.x / A.tiles_x;
    x0 = xt * 2 * P;
    if (A.axis == 1) {
      stride = A.nx;
      base = x0 + (long long)o * A.nx * A.ny;
      if (A.ndim == 3 && o == 0) {   // z = 0 plane: boundary, stays zero
        count_step(A);
        return;
      }
    } else {
      stride = A.nx * A.ny;
      base = x0 + (long long)o * A.nx;
      if (o == 0) {                  // y = 0 row: boundary, stays zero
        count_step(A);
        return;
      }
    }
  }

  // ---- constant tables (before the dependency wait): twiddles, and for the spectral ops the tables of
  // the transformed axis and the per-pencil values of the other axes
  {
    const float4* src = reinterpret_cast<const float4*>(A.tw);
    float4* dst = reinterpret_cast<float4*>(tab);
    for (int i = tid; i < SPLIT_TWN / 2; i += NT) cp_async<16>(&dst[i], &src[i]);
  }
  if constexpr (SplitOp<OP>::SPECTRAL) {
    const int la = A.axis;
    for (int i = tid; i < N; i += NT) {
      cp_async<4>(&tz[i], &A.zeta[la][i]);
      cp_async<4>(&te[i], &A.ex[la][i]);
      cp_async<4>(&tc[i], &A.ec[la][i]);
    }
    for (int i = tid; i < 2 * P; i += NT) {
      float z = A.zeta[0][x0 + i], e = A.ex[0][x0 + i], c = A.ec[0][x0 + i];
      if (A.ndim == 3) {
        z += A.zeta[1][o];
        e *= A.ex[1][o];
        c *= A.ec[1][o];
      }
      qz[i] = z;
      qe[i] = e;
      qc[i] = c;
    }
  }
  griddep_wait();
  if (A.step_inc && blockIdx.x == 0 && tid == 0) atomicAdd(A.step_inc, 1ULL);

  // ---- tile load / store
  auto buf = [&](int set, int p) -> C* { return bufs + (set * P + p) * LPS; };
  // contiguous rows: pair q = rows 2q, 2q+1; 16-byte loads staged in registers, then interleaved
  auto load_rows = [&](const float* __restrict__ src, int set) {
    constexpr int PER = N / 4;
    constexpr int CNT = (2 * PER + 159) / 160;   // vectors per thread at P = 2 (160 threads), rounded up
    const int items = P * PER;
    float4 va[CNT], vb[CNT];
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
      const int it = tid + c * NT;
      const int p = it / PER, k = it % PER, q = q0 + p;
      if (it < items && q < A.npairs) {
        va[c] = reinterpret_cast<const float4*>(src + (size_t)(2 * q) * A.nx)[k];
        vb[c] = reinterpret_cast<const float4*>(src + (size_t)(2 * q + 1) * A.nx)[k];
      } else {
        va[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        vb[c] = va[c];
      }
    }
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
      const int it = tid + c * NT;
      if (it < items) {
        C* b = buf(set, it / PER);
        const int j = 4 * (it % PER);
        b[sslot(j)] = j == 0 ? C{0.f, 0.f} : C{va[c].x, vb[c].x};   // position 0: boundary / mode 0
        b[sslot(j + 1)] = C{va[c].y, vb[c].y};
        b[sslot(j + 2)] = C{va[c].z, vb[c].z};
        b[sslot(j + 3)] = C{va[c].w, vb[c].w};
      }
    }
  };
  auto store_rows = [&](int set, float* __restrict__ dst, int t0, int nt) {
    constexpr int PER = N / 4;
    for (int it = tid - t0; it < P * PER; it += nt) {
      const int p = it / PER, k = it % PER, q = q0 + p;
      if (q >= A.npairs) continue;
      const C* b = buf(set, p);
      const int j = 4 * k;
      const C c0 = b[sslot(j)], c1 = b[sslot(j + 1)], c2 = b[sslot(j + 2)], c3 = b[sslot(j + 3)];
      reinterpret_cast<float4*>(dst + (size_t)(2 * q) * A.nx)[k] = make_float4(c0.x, c1.x, c2.x, c3.x);
      reinterpret_cast<float4*>(dst + (size_t)(2 * q + 1) * A.nx)[k] = make_float4(c0.y, c1.y, c2.y, c3.y);
    }
  };
  // strided columns: pair p = columns x0 + 2p, x0 + 2p + 1 of every row j (one 8-byte copy each)
  auto load_cols = [&](const float* __restrict__ src, int set) {
    for (int it = tid; it < P * N; it += NT) {
      const int p = it % P, j = it / P;
      if (j == 0) buf(set, p)[0] = C{0.f, 0.f};   // position 0: boundary / mode 0
      else cp_async<8>(buf(set, p) + sslot(j), src + (size_t)base + (size_t)j * stride + 2 * p);
    }
  };
  auto store_cols = [&](int set, float* __restrict__ dst, int t0, int nt) {
    for (int it = tid - t0; it < P * N; it += nt) {
      const int p = it % P, j = it / P;
      const C c = buf(set, p)[sslot(j)];
      *reinterpret_cast<float2*>(dst + (size_t)base + (size_t)j * stride + 2 * p) = make_float2(c.x, c.y);
    }
  };
  // dense user rows (ENTRY / EXIT): interior rows only, x = 1..N-1 at dense column x - 1
  auto dense_row = [&](int r) -> long long {
    const int y = r % A.ny, z = r / A.ny;
    if (y == 0 || (A.ndim == 3 && z == 0)) return -1;
    const long long dr = (A.ndim == 3 ? (long long)(z - 1) * (A.ny - 1) : 0LL) + (y - 1);
    return dr * (A.nx - 1);
  };
  auto load_dense = [&](const float* __restrict__ src, int set) {
    for (int it = tid; it < P * N; it += NT) {
      const int p = it / N, x = it % N, q = q0 + p;
      long long ra = -1, rb = -1;
      if (q < A.npairs) {
        ra = dense_row(2 * q);
        rb = dense_row(2 * q + 1);
      }
      const float a = (x >= 1 && ra >= 0) ? src[ra + x - 1] : 0.f;
      const float b = (x >= 1 && rb >= 0) ? src[rb + x - 1] : 0.f;
      buf(set, p)[sslot(x)] = C{a, b};
    }
  };
  auto store_dense = [&](int set, float* __restrict__ dst) {
    for (int it = tid; it < P * N; it += NT) {
      const int p = it / N, x = it % N, q = q0 + p;
      if (x == 0 || q >= A.npairs) continue;
      const long long ra = dense_row(2 * q), rb = dense_row(2 * q + 1);
      const C c = buf(set, p)[sslot(x)];
      if (ra >= 0) dst[ra + x - 1] = c.x;
      if (rb >= 0) dst[rb + x - 1] = c.y;
    }
  };

  // ---- loads
  if constexpr (OP == OP_ENTRY) load_dense(A.in0, 0);
  else if (contiguous) load_rows(A.in0, 0);
  else load_cols(A.in0, 0);
  if constexpr (NB == 2) load_cols(A.in1, 1);
  // position N of every buffer is read by the gathers and stays 0
  for (int i = tid; i < NB * P; i += NT) bufs[i * LPS + sslot(N)] = C{0.f, 0.f};
  cp_async_wait_all();
  __syncthreads();

  // ---- warp roles: field set f, pair group g (pairs 2g, 2g+1), role 0/1 A of pair 0/1, 2/3 C of pair
  // 0/1, 4 B of both
  const int wpf = 5 * (P / 2);
  const int f = warp / wpf, wi = warp % wpf, g = wi / 5, role = wi % 5;
  C* const wscr = scr + warp * SPLIT_SCR;
  const float hsc = A.sc, fl = A.flin, fc = A.fcub;
  const int fs = f < NB ? f : 0;
  // The passes of one kernel run their transforms through a single call site (the loop below), so that
  // the transform code exists once per kernel.
  constexpr int NT_TR = SplitOp<OP>::SPECTRAL ? 2 : (OP == OP_REACT ? 2 : 1);
#pragma unroll 1
  for (int t = 0; t < NT_TR; ++t) {
    bool active = true;
    if constexpr (SplitOp<OP>::SPECTRAL) {
      if (t == 0) {
        active = f < NF;
      } else {
        // stage combination, mode by mode, between the forward and the inverse transform
        __syncthreads();
        split_epilogue<OP>(A, P, bufs, tz, te, tc, qz, qe, qc, x0, tid, NT);
        __syncthreads();
        active = f == 0;
        if constexpr (OP == OP_S1) {
          if (f == 1) store_cols(1, A.out1, NT / 2, NT / 2);   // P, while set 0 transforms back
        }
      }
    }
    split_dst_group(role, lane, buf(fs, 2 * g), buf(fs, 2 * g + 1), tab, wscr, active, OP == OP_REACT && t == 0,
                    fl, fc, hsc);
  }
  __syncthreads();

  griddep_launch_dependents();
  if constexpr (OP == OP_EXIT) store_dense(0, A.out0);
  else if (contiguous) store_rows(0, A.out0, 0, NT);
  else store_cols(0, A.out0, 0, NT);
}

}  // namespace etd
