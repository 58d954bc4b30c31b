// pass_kernel.cuh - one "axis pass" of the fast EIFE solve (Section 4): a CTA stages a tile of
// pencils of one axis in shared memory, runs a short program of DST-I transforms (DHT on periodic
// axes, template variant V_HART) with fused pointwise epilogues, and writes the tile back.
//
// Homogeneous Dirichlet: index 0 of each pitched axis is the boundary node / sine mode 0 and stays
// zero; the dense user field holds the N_a - 1 interior nodes. Periodic (V_HART kernels; a plan's
// axes are all periodic or all Dirichlet): every index 0..N_a-1 is a node / Hartley mode and the
// dense field is the pitched field itself.
//
// Pencil pairs: along x (contiguous rows) a pair is two adjacent rows; along y or z (strided) a
// pair is two adjacent x-columns, so each row segment of the tile is already a complex pair.
//
// Ops and what they compute (U physical, ~ spectral along the transformed axes):
//   ENTRY     dense u -> pitched field, DST along x                              (x)
//   EXIT      DST along x -> dense u                                             (x)
//   PACK/UNPACK  dense <-> pitched without transform                             (x)
//   REACT     DST, nodal reaction f(u) = flin u + fcub u^3 [+ flog artanh u], DST (x)
//   TRANSFORM DST                                                                (any axis)
//   RK1       last axis: DST(U), DST(N0), U~+ = e^{-z} U~ + tau phi1(-z) N0~, DST  -> eq. (2.13)
//   S1        last axis: DST(U), DST(N0), U2~ = e^{-c2 z} U~ + c2 tau phi1(-c2 z) N0~ (DST -> out0),
//             P = e^{-z} U~ + tau (phi1 - phi2/c2)(-z) N0~ (-> out1)               -> eq. (2.14)
//   S2        last axis: DST(N2), U~+ = P + tau/c2 phi2(-z) N2~, DST               -> eq. (2.14)
// with z = tau D (mu_x + mu_y [+ mu_z]) per mode (the tensor H of Section 4 times tau).
// Plans that keep the state also in its fully spectral form U~ (the last-axis DST of U, written by
// the step's last pass) run the stage passes without the forward DST of U:
//   RK1S      last axis: in U~, N0; DST(N0), U~+ (-> out1), DST -> U+ (out0)
//   S1S       last axis: in U~, N0; DST(N0), U2~ and P as S1 (P -> out1), DST -> U2 (out0)
//   S2S       last axis: as S2, and U~+ (-> out1) before the closing DST
#pragma once
#include <type_traits>

#include "dst_engine.cuh"
#include "etd_coeffs.cuh"

namespace etd {

enum PassOp : int {
  OP_ENTRY = 0,
  OP_EXIT = 1,
  OP_REACT = 2,
  OP_TRANSFORM = 3,
  OP_RK1 = 4,
  OP_S1 = 5,
  OP_S2 = 6,
  OP_PACK = 7,
  OP_UNPACK = 8,
  OP_RK1S = 9,
  OP_S1S = 10,
  OP_S2S = 11,
  OP_COUNT = 12,
};

enum EpiKind : int { EPI_PLAIN = 0, EPI_REACT = 1, EPI_RK1 = 2, EPI_S1 = 3, EPI_S2 = 4 };

// f(u) = flin u + fcub u^3 + flog artanh(u); flog artanh u = (flog/2) ln((1+u)/(1-u)) is the
// Flory-Huggins term of Example 5.3 (Section 5.2).
__device__ __forceinline__ float artanh_(float v) { return atanhf(v); }
__device__ __forceinline__ double artanh_(double v) { return atanh(v); }

template <class T> struct PassArgs {
  int op, axis, ndim;
  int nx, ny, nz;   // pitched extents; nz = 1 in 2D. Index 0 of each axis is the boundary / mode 0.
  int P;            // pencil pairs per CTA
  int lp;           // complex slots per pair in shared memory (>= the layout minimum)
  int tiles_x;      // strided passes: nx / (2P)
  int npairs;       // contiguous passes: ny * nz / 2
  int user_slot;    // batched entry/exit passes: index of the caller's field pointer, else -1
  const T* in0;
  const T* in1;
  T* out0;
  T* out1;
  const T* tw;      // exp(2 pi i m / M), m < M (M = FFT length), interleaved (re, im)
  const T* sn;      // sin(pi j / N), j < N (recurrence variant only)
  const T* zeta[3]; // per paper axis: tau D mu_a
  const T* ex[3];   // exp(-tau D mu_a)
  const T* ec[3];   // exp(-c2 tau D mu_a)
  T sc, tau, c2, flin, fcub, flog;
  // Separable time-dependent source of the reaction (REACT passes; src_gx == NULL: none). The pass
  // stores S_x f(u), so it adds src_amp exp(-src_rate t) (S_x g_x)[k] g_y[y] g_z[z] at node row
  // (y, z) and x mode k, t = t0 + (steps + src_c) tau.
  const T* src_gx;                       // [nx] spectral x profile S_x g_x (Dirichlet: mode 0 = 0)
  const T* src_gy;                       // [ny] nodal y profile (Dirichlet: boundary 0)
  const T* src_gz;                       // [nz] nodal z profile (3D; NULL in 2D)
  const double* src_t0;                  // start time of the run
  const unsigned long long* step_ctr;    // time steps completed in the run
  unsigned long long* step_inc;          // the last pass of a step counts it (NULL: no)
  double src_amp, src_rate, src_c;
  // Per-mode phi-function weights of the last-axis passes of FP32 2D plans (NULL: evaluated in the
  // kernel), [y mode][x mode]: S1 float2 {c2 tau phi1(-c2 z), tau (phi1 - phi2/c2)(-z)}, S2 float
  // tau phi2(-z)/c2, RK1 float tau phi1(-z).
  const T* coef;
  int coef_smem;    // 1: the kernel stages its tile's weights in shared memory before the dependency wait
                    // (set by the host for the lengths that do, TABLES_STAGED)
};

// Asynchronous global -> shared copies (cp.async): every load of a tile is in flight at once and
// the CTA waits a single time, instead of one memory latency per register-staged loop iteration.
template <int B> __device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

// FP32 kernels whose transforms fit are held to 64 registers (two 512-thread CTAs per SM), so that
// twice as many warps hide shared-memory and FMA latency; the others keep 128.
template <class T, int N, int VAR> constexpr int pass_min_blocks();
// Kernels compiled with the table epilogue (per-mode weight tables of FP32 2D plans): the FP32 ones with
// the full register budget.
template <class T, int N, int VAR> constexpr bool TABLES_ON() { return sizeof(T) == 4 && pass_min_blocks<T, N, VAR>() == 1; }
// Of those, the lengths whose tile leaves room for the tile's rows of the tables in shared memory
// (staged before the dependency wait; the host passes no tables where a launch cannot stage them);
// longer axes read the tables from global memory.
template <class T, int N, int VAR> constexpr bool TABLES_STAGED() { return TABLES_ON<T, N, VAR>() && N <= 1536; }
// Shapes with kernels per operation for the passes of a time step (REACT, TRANSFORM, RK1S, S1S, S2S):
// the FP32 lengths of the large 2D and 3D workloads and of batches of meshes from 64 to 384, and the FP64
// length of the 2D workloads (N = 1024).
template <class T, int N, int VAR> constexpr bool pass_op_kernels() {
  return (sizeof(T) == 4 &&
          ((VAR == V_ODD && (N == 1024 || N == 2048)) ||
           (VAR == V_REC && (N == 64 || N == 96 || N == 128 || N == 192 || N == 256 || N == 384)) ||
           (VAR == V_HART && N == 128))) ||
         (sizeof(T) == 8 && VAR == V_REC && N == 1024);
}
// FP64: the operation-fixed kernels (the 2D FP64 workloads' axis length) read the tables from global memory.
template <class T, int N, int VAR> constexpr bool TABLES_ANY() {
  return TABLES_ON<T, N, VAR>() || (sizeof(T) == 8 && pass_op_kernels<T, N, VAR>());
}

// Per-mode weights of one pencil pair at table position m: S1 four values (two per pencil), S2 and RK1
// two (one per pencil), loaded as 16-byte vectors.
template <class T> struct PairWeights;
template <> struct PairWeights<float> {
  using W4 = float4;
  using W2 = float2;
  static __device__ __forceinline__ W4 ld4(const float* p, size_t m) { return reinterpret_cast<const float4*>(p)[m]; }
  static __device__ __forceinline__ W2 ld2(const float* p, size_t m) { return reinterpret_cast<const float2*>(p)[m]; }
};
template <> struct PairWeights<double> {
  struct W4 { double x, y, z, w; };
  using W2 = double2;
  static __device__ __forceinline__ W4 ld4(const double* p, size_t m) {
    const double2 a = reinterpret_cast<const double2*>(p)[2 * m], b = reinterpret_cast<const double2*>(p)[2 * m + 1];
    return W4{a.x, a.y, b.x, b.y};
  }
  static __device__ __forceinline__ W2 ld2(const double* p, size_t m) { return reinterpret_cast<const double2*>(p)[m]; }
};
template <class T, int N, int VAR> constexpr int pass_min_blocks() {
  // 3 x 2^k lengths above 48 keep 128 registers (their radix-3/12 stages spill at 64), except the
  // recurrence plan of N = 96 (radices 4, 3, 8), which fits
  return (sizeof(T) == 4 && N <= 512 && (N % 3 != 0 || N <= 48 || (N == 96 && VAR == V_REC))) ? 2 : 1;
}
// The last pass of a time step counts it, in CTA 0, after the dependency wait (the step's reaction
// passes, which read the count, have completed then). CTAs that return early (boundary tiles) call
// this on their way out.
template <class T> __device__ __forceinline__ void count_step(const PassArgs<T>& A) {
  if (A.step_inc && blockIdx.x == 0 && threadIdx.x == 0) {
    griddep_wait();
    atomicAdd(A.step_inc, 1ULL);
  }
}

// OPC: the pass operation fixed at compile time (one of PassOp), or -1 to take it from A.op. A kernel
// with a fixed operation holds only that operation's code, so the instructions a launch executes lie
// together (fewer instruction-cache misses than in the kernel that serves every operation).
template <class T, int N, int VAR, int OPC = -1>
__device__ __forceinline__ void pass_body(const PassArgs<T>& A, const int tile) {
  using L = PairLayout<T, N, VAR>;
  constexpr bool PER = L::HART;   // periodic: no boundary planes, rows or slots
  using C = Cx<T>;
  using VT = typename V2<T>::type;
  constexpr int TPP = L::TPP;
  const int LP = A.lp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // shared memory: per-pass twiddle tables, then the tile buffers, then scan scratch
  constexpr int TWN = L::TWN > 0 ? L::TWN : 1;
  C* tws = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = tws;
  const T* __restrict__ sn = A.sn;
  C* b0 = tws + ((TWN + 1) & ~1);
  const int op = OPC >= 0 ? OPC : A.op;
  const bool two = (op == OP_RK1 || op == OP_S1 || op == OP_S2 || op == OP_RK1S || op == OP_S1S || op == OP_S2S);
  C* b1 = b0 + A.P * LP;
  C* scr = b0 + (two ? 2 : 1) * A.P * LP;
  // spectral passes (two buffers) also stage the transformed axis's e, ec, zeta tables (3 N values);
  // a pass that stages its weight tables (A.coef_smem) leaves zeta out (the table epilogue does not
  // read it) and puts the weights at the next 16-byte boundary instead
  T* te = reinterpret_cast<T*>(scr + A.P * (TPP > 32 ? TPP / 32 : 1));
  T* tcs = te + N;
  T* tz = tcs + N;
  T* tco = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(tz) + 15) & ~(uintptr_t)15);
  const int tid = threadIdx.x, NT = blockDim.x;
  const int P = A.P;
  const int p = tid / TPP, l = tid % TPP;
  const bool contiguous = (A.axis == 0);

  // ---- tile geometry
  int q0 = 0, stride = 0, x0 = 0, o = 0;
  long long base = 0;
  if (contiguous) {
    q0 = tile * P;
  } else {
    const int W = 2 * P;
    const int xt = tile % A.tiles_x;
    o = tile / A.tiles_x;
    x0 = xt * W;
    if (A.axis == 1) {
      stride = A.nx;
      base = x0 + (long long)o * A.nx * A.ny;
      if (!PER && A.ndim == 3 && o == 0) {   // z = 0 plane: boundary, stays zero
        count_step(A);
        return;
      }
    } else {
      stride = A.nx * A.ny;
      base = x0 + (long long)o * A.nx;
      if (!PER && o == 0) {                  // y = 0 row: boundary, stays zero
        count_step(A);
        return;
      }
    }
  }

  // ---- tile load / store helpers
  const int spp = tid % P, sj0 = tid / P;   // strided tiles: pair and first row of this thread
  // Tile load of one field into buf. Strided passes: cp.async of one complex pair (two adjacent
  // x values) per (row j, pair pp); a thread keeps its pair index and walks rows, so no division.
  // Contiguous passes: 16-byte loads of both rows of a pair staged in registers (all issued before
  // the first shared store), interleaved into complex slots.
  constexpr int V = (sizeof(T) == 4 && N % 4 == 0) ? 4 : 2;   // elements per vector load
  using VL = typename std::conditional<V == 4, float4, VT>::type;
  auto load_tile = [&](const T* __restrict__ src, C* buf) {
    if (contiguous) {
      constexpr int PER = N / V;                               // vectors per row
      constexpr int CNT = (PER + TPP - 1) / TPP;               // per thread and row
      const int q = q0 + p;
      C* bpp = buf + p * LP;
      if (q < A.npairs) {
        const VL* ra = reinterpret_cast<const VL*>(src + (size_t)(2 * q) * A.nx);
        const VL* rb = reinterpret_cast<const VL*>(src + (size_t)(2 * q + 1) * A.nx);
        VL va[CNT], vb[CNT];
#pragma unroll
        for (int c = 0; c < CNT; ++c) {
          const int k = l + c * TPP;
          if (PER % TPP == 0 || k < PER) {
            va[c] = ra[k];
            vb[c] = rb[k];
          }
        }
#pragma unroll
        for (int c = 0; c < CNT; ++c) {
          const int k = l + c * TPP;
          if (PER % TPP == 0 || k < PER) {
            const T* a = reinterpret_cast<const T*>(&va[c]);
            const T* b = reinterpret_cast<const T*>(&vb[c]);
#pragma unroll
            for (int e = 0; e < V; ++e) bpp[L::at(V * k + e)] = C{a[e], b[e]};
          }
        }
      } else {
        for (int j = l; j < N; j += TPP) bpp[L::at(j)] = C{T(0), T(0)};
      }
    } else {
      // thread = (pair pp, first row j0); rows j0 + k*TPP, k < N/TPP (N/TPP is exact)
      C* sd = buf + spp * LP;
      const T* gs = src + (size_t)base + (size_t)sj0 * stride + 2 * spp;
      const size_t gstep = (size_t)TPP * stride;
      const int atj0 = L::at(sj0);
#pragma unroll
      for (int k = 0; k < N / TPP; ++k)
        cp_async<2 * sizeof(T)>(sd + L::at_stride(atj0, sj0, k), gs + k * gstep);
    }
  };
  auto store_tile = [&](const C* buf, T* __restrict__ dst) {
    if (contiguous) {
      constexpr int PER = N / V;
      const int q = q0 + p;
      if (q < A.npairs) {
        const C* bpp = buf + p * LP;
        VL* ra = reinterpret_cast<VL*>(dst + (size_t)(2 * q) * A.nx);
        VL* rb = reinterpret_cast<VL*>(dst + (size_t)(2 * q + 1) * A.nx);
        for (int k = l; k < PER; k += TPP) {
          VL va, vb;
          T* a = reinterpret_cast<T*>(&va);
          T* b = reinterpret_cast<T*>(&vb);
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const C c = bpp[L::at(V * k + e)];
            a[e] = c.x;
            b[e] = c.y;
          }
          ra[k] = va;
          rb[k] = vb;
        }
      }
    } else {
      const C* sd = buf + spp * LP;
      T* gd = dst + (size_t)base + (size_t)sj0 * stride + 2 * spp;
      const size_t gstep = (size_t)TPP * stride;
      const int atj0 = L::at(sj0);
#pragma unroll
      for (int k = 0; k < N / TPP; ++k) {
        const C c = sd[L::at_stride(atj0, sj0, k)];
        *reinterpret_cast<VT*>(gd + k * gstep) = VT{c.x, c.y};
      }
    }
  };
  // dense user layout: rows of nx-1 interior values, only rows with y >= 1 (and z >= 1 in 3D);
  // periodic: the pitched layout itself
  auto dense_row = [&](int r) -> long long {
    if constexpr (PER) return (long long)r * A.nx;
    const int y = r % A.ny, z = r / A.ny;
    if (y == 0 || (A.ndim == 3 && z == 0)) return -1;
    const long long dr = (A.ndim == 3 ? (long long)(z - 1) * (A.ny - 1) : 0LL) + (y - 1);
    return dr * (A.nx - 1);
  };
  // dense rows of this thread's pair (computed once); -1 for boundary rows or pairs past the end
  long long dra = -1, drb = -1;
  if (op == OP_ENTRY || op == OP_EXIT || op == OP_PACK || op == OP_UNPACK) {
    const int q = q0 + p;
    if (q < A.npairs) {
      dra = dense_row(2 * q);
      drb = dense_row(2 * q + 1);
    }
  }
  auto load_dense = [&](const T* __restrict__ src, C* buf) {
    C* bpp = buf + p * LP;
    constexpr int X0 = PER ? 0 : 1;   // dense column of pitched index x is x - X0
    for (int x = l; x < N; x += TPP) {
      const T a = (x >= X0 && dra >= 0) ? src[dra + x - X0] : T(0);
      const T b = (x >= X0 && drb >= 0) ? src[drb + x - X0] : T(0);
      bpp[L::at(x)] = C{a, b};
    }
  };
  auto store_dense = [&](const C* buf, T* __restrict__ dst) {
    const C* bpp = buf + p * LP;
    constexpr int X0 = PER ? 0 : 1;
    for (int x = l + (l < X0 ? TPP : 0); x < N; x += TPP) {
      const C c = bpp[L::at(x)];
      if (dra >= 0) dst[dra + x - X0] = c.x;
      if (drb >= 0) dst[drb + x - X0] = c.y;
    }
  };

  // ---- loads (twiddles of the transformed axis: constant tables, issued before the dependency
  // wait; then the tile, produced by the previous kernel)
  if (op != OP_PACK && op != OP_UNPACK) {
    const C* gtw = reinterpret_cast<const C*>(A.tw);
    for (int i = tid; i < L::TWN; i += NT) cp_async<2 * sizeof(T)>(&tws[i], &gtw[i]);
  }
  const bool coef_smem = TABLES_STAGED<T, N, VAR>() && two && A.coef;
  if (two) {
    // the transformed axis's tables, selected without indexing the descriptor's arrays by a run-time
    // value (which would keep a batched kernel's copy of the descriptor in local memory)
    const int ax = A.axis;
    const T* gz = ax == 0 ? A.zeta[0] : (ax == 1 ? A.zeta[1] : A.zeta[2]);
    const T* ge = ax == 0 ? A.ex[0] : (ax == 1 ? A.ex[1] : A.ex[2]);
    const T* gc = ax == 0 ? A.ec[0] : (ax == 1 ? A.ec[1] : A.ec[2]);
    for (int i = tid; i < N; i += NT) {
      if (!coef_smem) cp_async<sizeof(T)>(&tz[i], &gz[i]);
      cp_async<sizeof(T)>(&te[i], &ge[i]);
      cp_async<sizeof(T)>(&tcs[i], &gc[i]);
    }
  }
  if (coef_smem) {
    // rows j < N of the tile's 2P x modes, fpm floats per mode, as 16-byte chunks stored chunk-major
    // ([chunk c][row j]: the lanes of a warp, consecutive j, then read consecutive chunks)
    const int fpm = (op == OP_S1 || op == OP_S1S) ? 2 : 1;
    const int cpr = 2 * A.P * fpm / 4;
    for (int i = tid; i < N * cpr; i += NT) {
      const int j = i / cpr, c = i - j * cpr;
      cp_async<16>(tco + ((size_t)c * N + j) * 4, A.coef + ((size_t)j * A.nx + x0) * fpm + 4 * c);
    }
  }
  griddep_wait();
  if (A.step_inc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.step_inc, 1ULL);
  if (op == OP_ENTRY || op == OP_PACK) {
    load_dense(A.in0, b0);
  } else {
    load_tile(A.in0, b0);
    if (two) load_tile(A.in1, b1);
  }
  cp_async_wait_all();
  __syncthreads();

  if (op == OP_PACK) {
    store_tile(b0, A.out0);
    return;
  }
  if (op == OP_UNPACK) {
    store_dense(b0, A.out0);
    return;
  }

  // ---- per-pencil constants of the spectral epilogues (last axis passes only)
  const int la = A.axis;  // transformed axis
  T pz[2] = {T(0), T(0)}, pe[2] = {T(1), T(1)}, pc[2] = {T(1), T(1)};
  const T* zj = tz;   // staged copies of A.zeta[la], A.ex[la], A.ec[la]
  const T* ej = te;
  const T* cj = tcs;
  if (two) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int x = x0 + 2 * p + s;
      pz[s] = A.zeta[0][x];
      pe[s] = A.ex[0][x];
      pc[s] = A.ec[0][x];
      if (A.ndim == 3) {
        pz[s] += A.zeta[1][o];
        pe[s] *= A.ex[1][o];
        pc[s] *= A.ec[1][o];
      }
    }
  }

  // ---- DST program: transforms s0 .. nd-1 of buffer bsel[s], each followed by epilogue epi[s]; the
  // passes with a spectral input (RK1S, S1S) start after the forward DST of U
  int nd = 0, s0 = 0, bsel[3] = {0, 0, 0}, epi[3] = {EPI_PLAIN, EPI_PLAIN, EPI_PLAIN};
  switch (op) {
    case OP_ENTRY: case OP_EXIT: case OP_TRANSFORM: nd = 1; break;
    case OP_REACT: nd = 2; break;   // the reaction is applied as the second transform reads
    case OP_RK1: case OP_RK1S: nd = 3; bsel[1] = 1; epi[1] = EPI_RK1; break;
    case OP_S1: case OP_S1S: nd = 3; bsel[1] = 1; epi[1] = EPI_S1; break;
    case OP_S2: case OP_S2S: nd = 2; epi[0] = EPI_S2; break;
    default: break;
  }
  if (op == OP_RK1S || op == OP_S1S) s0 = 1;
  // Second outputs, stored with the first at the end from b1: P (S1, S1S: b1 is not touched after the
  // stage epilogue) and U~+ (RK1S, S2S: the stage epilogue writes its result to b1 as well, whose
  // contents, N0~ or P, it no longer needs, before the closing DST of b0).
  const bool out1_b1 = (op == OP_S1 || op == OP_S1S || op == OP_RK1S || op == OP_S2S);
  const bool mirror = (op == OP_RK1S || op == OP_S2S);
  C* const b0p = b0 + p * LP;
  C* const b1p = b1 + p * LP;
  C* const scrp = scr + p * (TPP > 32 ? TPP / 32 : 1);
  const T tau = A.tau, c2 = A.c2, inv_c2 = T(1) / A.c2;

  auto epilogue = [&](int kind, int j, C w) -> C {
    const T zjj = zj[j], ejj = ej[j];
    T out[2];
    const T wv[2] = {w.x, w.y};
    // phi_k(-zeta) in closed form for zeta >= 1 from one reciprocal per mode; the series runs only
    // in warps holding a mode below zeta = 1 (or c2 zeta = 1), the low-mode corner of the spectrum
    // (every lane of the warp votes with its own predicate, so a lane that needs it gets it).
    const unsigned act = __activemask();
    if (kind == EPI_RK1) {
      const C u = b0p[L::at(j)];
      const T uv[2] = {u.x, u.y};
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const T zeta = pz[t] + zjj, E = pe[t] * ejj;
        T p1, p2, rz;
        stage_phi12<T>(zeta, E, act, p1, p2, rz);
        out[t] = E * uv[t] + tau * p1 * wv[t];
      }
      b0p[L::at(j)] = C{out[0], out[1]};
      return mirror ? C{out[0], out[1]} : w;   // (written to b1, the buffer transformed last)
    }
    if (kind == EPI_S1) {
      const T cjj = cj[j];
      const C u = b0p[L::at(j)];
      const T uv[2] = {u.x, u.y};
      T u2[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const T zeta = pz[t] + zjj, E = pe[t] * ejj, Ec = pc[t] * cjj;
        T p1, p2, rz;
        stage_phi12<T>(zeta, E, act, p1, p2, rz);
        const T t1 = tau * stage_phi1c<T>(zeta, Ec, c2, rz, act);   // c2 tau phi1(-c2 zeta)
        u2[t] = Ec * uv[t] + t1 * wv[t];
        out[t] = E * uv[t] + tau * (p1 - p2 * inv_c2) * wv[t];
      }
      b0p[L::at(j)] = C{u2[0], u2[1]};
      return C{out[0], out[1]};
    }
    // EPI_S2: P from the second buffer
    const C pp = b1p[L::at(j)];
    const T pv[2] = {pp.x, pp.y};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const T zeta = pz[t] + zjj, E = pe[t] * ejj;
      T p1, p2, rz;
      stage_phi12<T>(zeta, E, act, p1, p2, rz);
      out[t] = pv[t] + (tau * inv_c2) * p2 * wv[t];
    }
    if (mirror) b1p[L::at(j)] = C{out[0], out[1]};
    return C{out[0], out[1]};
  };

  // 2D plans: the phi-function weights of the stage combination come from per-mode tables of FP64
  // values (FP32 plans: rounded once) (A.coef, [y mode][x mode]; e^{-z}, e^{-c2 z} are products of the
  // per-axis factors), with every table load of a chunk of positions issued before the first use. Same
  // effect on the buffers as the epilogue above.
  // Compiled into the FP32 kernels with the full register budget and the FP64 operation-fixed kernels
  // only; the others evaluate the weights.
  constexpr bool TABLES = TABLES_ANY<T, N, VAR>();
  auto table_epilogue = [&](int kind, C* bpk) {
    if constexpr (TABLES) {
      constexpr int CNT = (N + TPP - 1) / TPP, CH = sizeof(T) == 4 ? 4 : 2;
      using PW = PairWeights<T>;
      const size_t col = (size_t)x0 + 2 * p;
#pragma unroll
      for (int c0 = 0; c0 < CNT; c0 += CH) {
        typename PW::W4 cf4[CH];
        typename PW::W2 cf2[CH];
        if constexpr (TABLES_STAGED<T, N, VAR>()) {   // staged chunk-major: S1 one pair per chunk, else two
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int j = l + (c0 + c) * TPP;
            if (c0 + c < CNT && j < N) {
              if (kind == EPI_S1) cf4[c] = reinterpret_cast<const float4*>(tco)[p * N + j];
              else cf2[c] = reinterpret_cast<const float2*>(tco)[((p >> 1) * N + j) * 2 + (p & 1)];
            }
          }
        } else {           // the plan's [y mode][x mode] table
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int j = l + (c0 + c) * TPP;
            if (c0 + c < CNT && j < N) {
              const size_t m = ((size_t)j * A.nx + col) / 2;
              if (kind == EPI_S1) cf4[c] = PW::ld4(A.coef, m);
              else cf2[c] = PW::ld2(A.coef, m);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int j = l + (c0 + c) * TPP;
          if (c0 + c >= CNT || j >= N) continue;
          const int aj = L::at(j);
          const C w = bpk[aj];
          if (kind == EPI_S1) {          // {c2 tau phi1(-c2 z), tau (phi1 - phi2/c2)(-z)} per mode
            const C u = b0p[aj];
            b0p[aj] = C{pc[0] * cj[j] * u.x + cf4[c].x * w.x, pc[1] * cj[j] * u.y + cf4[c].z * w.y};
            bpk[aj] = C{pe[0] * ej[j] * u.x + cf4[c].y * w.x, pe[1] * ej[j] * u.y + cf4[c].w * w.y};
          } else if (kind == EPI_RK1) {  // tau phi1(-z) per mode
            const C u = b0p[aj];
            const C r{pe[0] * ej[j] * u.x + cf2[c].x * w.x, pe[1] * ej[j] * u.y + cf2[c].y * w.y};
            b0p[aj] = r;
            if (mirror) b1p[aj] = r;
          } else {                       // S2: tau phi2(-z)/c2 per mode; P in the second buffer
            const C pp = b1p[aj];
            const C r{pp.x + cf2[c].x * w.x, pp.y + cf2[c].y * w.y};
            bpk[aj] = r;
            if (mirror) b1p[aj] = r;
          }
        }
      }
      __syncthreads();
    }
  };
  auto stage_epilogue = [&](int kind, C* bpk) {
    if (TABLES && A.coef) table_epilogue(kind, bpk);
    else epilogue_pair<T, N, VAR>(bpk, l, [&](int j, C w) -> C { return epilogue(kind, j, w); });
  };

  // Odd-extension kernels with the full register budget (one CTA of 512 threads per SM) run the
  // two forward transforms of RK1/S1 (of U and of N0) together, sharing each Stockham pass's
  // barriers; under the halved budget the second set of butterfly registers would spill.
  if constexpr (L::ODD && pass_min_blocks<T, N, VAR>() == 1) {
    if (op == OP_RK1 || op == OP_S1) {
      C* const bps[2] = {b0p, b1p};
      C* const scrs[2] = {scrp, scrp};   // unused by the odd-extension variant
      dst_pairs<T, N, VAR, 2>(bps, tw, sn, l, scrs, A.sc);
      stage_epilogue(epi[1], b1p);
      s0 = 2;
    }
  }
  // A logarithmic reaction term (flog != 0; periodic kernels only, the Flory-Huggins reaction of
  // Example 5.3) takes an unfused pointwise pass over the nodal values before the second transform
  // of REACT; the Dirichlet kernels are compiled without it.
  const bool logr = PER && op == OP_REACT && A.flog != T(0);
#pragma unroll 1
  for (int s = s0; s < nd; ++s) {
    const int kind = epi[s];
    C* bp = bsel[s] ? b1p : b0p;
    if constexpr (PER) {
      if (logr && s == 1) {
        const T fl = A.flin, fc = A.fcub, fg = A.flog;
        epilogue_pair<T, N, VAR>(bp, l, [&](int, C w) -> C {
          return C{w.x * (fl + fc * w.x * w.x) + fg * artanh_(w.x), w.y * (fl + fc * w.y * w.y) + fg * artanh_(w.y)};
        });
      }
    }
    const React<T> rx{op == OP_REACT && s == 1 && !logr, A.flin, A.fcub};
    dst_pair<T, N, VAR>(bp, tw, sn, l, scrp, A.sc, rx);
    if (kind != EPI_PLAIN) stage_epilogue(kind, bp);
  }

  if (op == OP_REACT && A.src_gx) {
    // separable source, already in the x-spectral form the pass stores (rare path)
    const int q = q0 + p;
    if (q < A.npairs) {
      const double t = *A.src_t0 + ((double)*A.step_ctr + A.src_c) * (double)A.tau;
      const double amp = A.src_amp * exp(-A.src_rate * t);
      const int ra = 2 * q, rb = 2 * q + 1;
      const double ga = amp * (double)A.src_gy[ra % A.ny] * (A.src_gz ? (double)A.src_gz[ra / A.ny] : 1.0);
      const double gb = amp * (double)A.src_gy[rb % A.ny] * (A.src_gz ? (double)A.src_gz[rb / A.ny] : 1.0);
      for (int j = l; j < N; j += TPP) {
        const double g = (double)A.src_gx[j];
        C v = b0p[L::at(j)];
        v.x += (T)(ga * g);
        v.y += (T)(gb * g);
        b0p[L::at(j)] = v;
      }
    }
    __syncthreads();
  }
  griddep_launch_dependents();
  if (op == OP_EXIT) store_dense(b0, A.out0);
  else store_tile(b0, A.out0);
  if (out1_b1) store_tile(b1, A.out1);
}

// One plan: the launch covers the tiles of one field.
template <class T, int N, int VAR>
__global__ void __launch_bounds__(512, pass_min_blocks<T, N, VAR>()) pass_kernel(const PassArgs<T> A) {
  pass_body<T, N, VAR>(A, (int)blockIdx.x);
}

// The same with the operation fixed (A.op must equal OPC).
template <class T, int N, int VAR, int OPC>
__global__ void __launch_bounds__(512, pass_min_blocks<T, N, VAR>()) pass_kernel_op(const PassArgs<T> A) {
  pass_body<T, N, VAR, OPC>(A, (int)blockIdx.x);
}

// Batches: one launch covers the tiles of many independent problems whose transformed axis has
// length N. CTA b works on tile map[b].y of the problem described by descs[map[b].x]; entry and exit
// passes take the caller's field pointer from user[descs[.].user_slot].
template <class T, int N, int VAR>
__global__ void __launch_bounds__(512, pass_min_blocks<T, N, VAR>())
    pass_kernel_batched(const PassArgs<T>* __restrict__ descs, const int2* __restrict__ map, T* const* __restrict__ user) {
  const int2 m = map[blockIdx.x];
  PassArgs<T> A = descs[m.x];
  if (A.user_slot >= 0) {
    if (A.op == OP_ENTRY || A.op == OP_PACK) A.in0 = user[A.user_slot];
    else A.out0 = user[A.user_slot];
  }
  pass_body<T, N, VAR>(A, m.y);
}

// The same with the operation fixed (every descriptor's op must equal OPC).
template <class T, int N, int VAR, int OPC>
__global__ void __launch_bounds__(512, pass_min_blocks<T, N, VAR>())
    pass_kernel_batched_op(const PassArgs<T>* __restrict__ descs, const int2* __restrict__ map, T* const* __restrict__) {
  const int2 m = map[blockIdx.x];
  // the descriptor is read in place (read-only global memory, reloaded where needed) rather than copied
  // into registers, which the stage passes cannot spare
  pass_body<T, N, VAR, OPC>(descs[m.x], m.y);
}

// Host-side description of one instantiation.
struct KernelInfo {
  const void* fn;
  const void* fn_batched;
  const void* fn_op[OP_COUNT];           // kernels with the operation fixed, by PassOp (NULL: use fn)
  const void* fn_batched_op[OP_COUNT];   // the same for batches (NULL: use fn_batched)
  int N;
  int tpp;
  int lp;
  int elem;   // sizeof(T)
  int fft_len;  // M: 2N (odd extension) or N (recurrence, Hartley)
  int odd;      // transform variant: V_ODD odd extension, V_REC recurrence, V_HART Hartley
  int padg;     // one padding slot every padg positions
  int twn;      // twiddle table entries
  int radix[4]; // Stockham radices (0-terminated)
  int min_blocks;  // CTAs per SM the register budget was compiled for
};

template <int... Rs> void radix_list(int* out, Radices<Rs...>) {
  const int r[] = {Rs...};
  for (int i = 0; i < 4; ++i) out[i] = i < (int)sizeof...(Rs) ? r[i] : 0;
}

template <class T, int N, int VAR> KernelInfo kernel_info() {
  using L = PairLayout<T, N, VAR>;
  KernelInfo k{reinterpret_cast<const void*>(&pass_kernel<T, N, VAR>),
               reinterpret_cast<const void*>(&pass_kernel_batched<T, N, VAR>),
               {},
               {},
               N, L::TPP, L::LP, (int)sizeof(T), L::M,
               VAR, L::PADG, L::TWN, {0, 0, 0, 0}, pass_min_blocks<T, N, VAR>()};
  if constexpr (pass_op_kernels<T, N, VAR>()) {
    // single plans run the stage passes on the spectral state (RK1S, S1S, S2S)
    k.fn_op[OP_REACT] = reinterpret_cast<const void*>(&pass_kernel_op<T, N, VAR, OP_REACT>);
    k.fn_op[OP_TRANSFORM] = reinterpret_cast<const void*>(&pass_kernel_op<T, N, VAR, OP_TRANSFORM>);
    k.fn_op[OP_RK1S] = reinterpret_cast<const void*>(&pass_kernel_op<T, N, VAR, OP_RK1S>);
    k.fn_op[OP_S1S] = reinterpret_cast<const void*>(&pass_kernel_op<T, N, VAR, OP_S1S>);
    k.fn_op[OP_S2S] = reinterpret_cast<const void*>(&pass_kernel_op<T, N, VAR, OP_S2S>);
    // batches (FP32) are 2D: TRANSFORM only at entry (the generic kernel)
    if constexpr (sizeof(T) == 4) {
    k.fn_batched_op[OP_REACT] = reinterpret_cast<const void*>(&pass_kernel_batched_op<T, N, VAR, OP_REACT>);
    k.fn_batched_op[OP_RK1S] = reinterpret_cast<const void*>(&pass_kernel_batched_op<T, N, VAR, OP_RK1S>);
    k.fn_batched_op[OP_S1S] = reinterpret_cast<const void*>(&pass_kernel_batched_op<T, N, VAR, OP_S1S>);
    k.fn_batched_op[OP_S2S] = reinterpret_cast<const void*>(&pass_kernel_batched_op<T, N, VAR, OP_S2S>);
    }
  }
  radix_list(k.radix, typename L::Plan::R{});
  return k;
}

// Pair stride for a tile of P pairs: the smallest value >= the layout minimum whose residue keeps
// the per-row tile loads of strided passes (P lanes per row, consecutive rows) on distinct banks.
inline int pair_stride(const KernelInfo& k, int P) {
  const int groups = 128 / (2 * k.elem);           // complex slots per 128-byte bank cycle
  int lp = k.lp;
  if (P >= groups) {
    if (lp % 2 == 0) ++lp;                         // odd stride: P lanes of one row on distinct banks
  } else {
    const int want = (groups / P) % groups;        // residue in [0, groups)
    lp += ((want - lp % groups) + groups) % groups;  // at most groups - 1 steps, no loop
  }
  return lp;
}

// shared memory bytes of a launch
inline size_t pass_smem_bytes(const KernelInfo& k, int P, int nbuf) {
  const size_t c = 2 * (size_t)k.elem;
  const size_t tw = (size_t)(((k.twn > 0 ? k.twn : 1) + 1) & ~1) * c;
  const size_t bufs = (size_t)nbuf * P * pair_stride(k, P) * c;
  const size_t scr = (size_t)P * (k.tpp > 32 ? k.tpp / 32 : 1) * c;
  const size_t tabs = nbuf == 2 ? 3 * (size_t)k.N * k.elem : 0;   // zeta, e, ec of the spectral passes
  return tw + bufs + scr + tabs;
}

}  // namespace etd
