// etd_api.cu - plan, executor and C ABI of the GB300 EIFE solver (declared in include/etd.h).
//
// A time step (Section 4 fast solve of eqs. (2.13)/(2.14)) is a fixed list of axis-pass kernel
// launches over plan-owned fields. The state between steps is the field transformed along every
// axis but the last, so each step needs one pass per axis per transform stage:
//   2D EIFE2: x REACT(V->N0) | y S1(V,N0 -> V2,P) | x REACT(V2->N2) | y S2(N2,P -> V)
//   2D EIFE1: x REACT(V->N0) | y RK1(V,N0 -> V)
//   3D EIFE2: y T(V->V2) | x REACT(V2->N0) | y T(N0) | z S1(V,N0 -> V2,P) | y T(V2) |
//             x REACT(V2->N2) | y T(N2) | z S2(N2,P -> V)
//   3D EIFE1: y T(V->V2) | x REACT(V2->N0) | y T(N0) | z RK1(V,N0 -> V)
// etd_run enters with x (and y) forward transforms of the dense field and leaves with the inverse
// ones. Steady-state step lists are captured once into a CUDA graph and replayed.
//
// GEMM routes (tensor-core transform passes, gemm_pass.cuh): the state is spectral along every
// axis; a stage is d inverse passes (the last one applying the reaction) and d forward passes (the
// last one applying the ETD combination), each pass contracting one axis and rotating the layout:
//   2D EIFE2: x V->T1 | y REACT T1->T2 | x T2->T1 | y S1(T1,V -> V2,P) | x | y REACT | x | y S2(.,P -> V)
//   3D: the same with x, y, z passes (six per stage).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/etd.h"
#include "boundary.cuh"
#include "gemm_pass.cuh"
#include "monitor.cuh"
#include "pass_kernel.cuh"
#include "split_pass.cuh"

namespace etd {
// registry of instantiated pass kernels (generated per (type, N) translation units)
const KernelInfo* find_pass_kernel(int elem, int N, int variant);
// tensor-core transform passes (gemm_inst.cu)
const GemmKernelInfo* find_gemm_kernel(int bn, int route);
// split-radix FP32 passes for axes of length 1024 (split_inst.cu), one kernel per PassOp
const void* find_split_kernel(int op);
}  // namespace etd

using namespace etd;

namespace {
thread_local std::string g_last_error;
}  // namespace

void etd_internal_set_error(const char* msg) { g_last_error = msg; }

namespace {

etd_status fail(etd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define ETD_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (e_ == cudaErrorMemoryAllocation)                                                          \
        return fail(ETD_ERR_OOM, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return fail(ETD_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                               \
  } while (0)

enum PassKind { PK_ENTRY_EXIT = 0, PK_REACT = 1, PK_TRANSFORM = 2, PK_S1 = 3, PK_S2 = 4, PK_RK1 = 5,
                PK_PACK = 6, PK_MONITOR = 7, PK_BOUNDARY = 8 };
const char* kPassKindNames[ETD_NUM_PASS_KINDS] = {"entry_exit", "x_react", "transform", "stage1_etdrk2",
                                                   "stage2_etdrk2", "stage_etdrk1", "pack", "monitor",
                                                   "boundary"};

struct Launch {
  const void* fn;
  dim3 grid, block;
  size_t smem;
  int kind;
  alignas(64) unsigned char args[sizeof(PassArgs<double>) > sizeof(GemmParams) ? sizeof(PassArgs<double>)
                                                                                : sizeof(GemmParams)];
  size_t args_size;
  double alg_bytes;  // algorithmic HBM bytes of this launch (fields read + written)
};

int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return (v && *v) ? atoi(v) : dflt;
}

bool supported_length(int64_t n) {
  if (n < 4 || n > 2048) return false;
  int64_t m = n;
  if (m % 3 == 0) m /= 3;
  return (m & (m - 1)) == 0 && m >= 2;
}

}  // namespace

struct etd_plan_s {
  int ndim = 2;
  int64_t N[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  double D = 0, tau = 0;
  int scheme = 2;
  etd_options opt{};
  int elem = 8;
  int odd[3] = {0, 0, 0};  // transform variant per axis: V_ODD, V_REC (DST-I) or V_HART (periodic)
  int split[3] = {0, 0, 0};  // FP32 axes of length 1024 on the split-radix kernels (split_pass.cuh)
  int periodic = 0;        // every axis periodic (Hartley kernels), else homogeneous Dirichlet
  int nx = 1, ny = 1, nz = 1;
  size_t nfield = 0;       // pitched elements per field
  int64_t unknowns = 0;    // unknowns (interior nodes; periodic: all nodes)
  int device = 0;
  int num_sms = 148;
  void* ws = nullptr;      // fields
  void* F[6] = {};         // V, N0, V2, P, N2, and (spec) V~: V transformed along the last axis
  bool spec = false;       // the step keeps V~ and runs the stage passes on it (RK1S, S1S, S2S)
  void* tables = nullptr;
  const void* tw[3] = {};
  const void* stw[3] = {};   // twiddle tables of the split-radix kernels (split axes)
  void* coef = nullptr;      // per-mode stage coefficients of the last-axis passes of 2D plans (plan's dtype)
  size_t coef_s1 = 0, coef_s2 = 0, coef_rk1 = 0;   // element offsets of the S1, S2, RK1 tables
  const void* sn[3] = {};
  const void* zeta[3] = {};
  const void* ex[3] = {};
  const void* ec[3] = {};
  double sc[3] = {};
  std::vector<Launch> step;   // one time step
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  void* host_dev = nullptr;   // device copy for etd_run_host
  double* mon_part = nullptr;
  long long* mon_bad = nullptr;
  double* mon_out = nullptr;
  int mon_blocks = 0;
  size_t ws_bytes = 0;
  bool src_on = false;        // separable time-dependent source set (FFT routes)
  void* src_tab = nullptr;    // gx [nx], gy [ny] (, gz [nz]) in the plan's dtype; Dirichlet: index 0 = 0
  void* clock = nullptr;      // unsigned long long steps completed, then double t0
  double src_amp = 0, src_rate = 0;
  int gemm = 0;               // 0: FFT routes; 1 + GemmRoute: tensor-core transform passes
  void* gtab = nullptr;       // sine (periodic: Hartley) matrices S_a (fp32 TF32-rounded, or bf16 hi and lo)
  const void* gS[3][2] = {};  // per axis: S (TF32) or S_hi, S_lo (BF16x3)
  int* dev_err = nullptr;     // set by a tensor-core pass whose wait ran out
  // nonhomogeneous Dirichlet data (etd_set_boundary)
  bool bnd_on = false;
  etd_boundary_fn bnd_fn = nullptr;
  void* bnd_ctx = nullptr;
  int64_t bnd_count = 0;
  double* bnd_host = nullptr;  // pinned: per stage, values [count] then time derivatives [count]
  double* bnd_dev = nullptr;   // device copy of bnd_host
  void* bnd_field = nullptr;   // pitched B field of the plan's dtype
  double* bnd_ia = nullptr;    // 1 / lambda^A per axis: [nx], [ny], [nz]
};

namespace {

template <class T>
void fill_common(const etd_plan_s* pl, PassArgs<T>& a) {
  memset(&a, 0, sizeof(a));
  a.user_slot = -1;
  a.ndim = pl->ndim;
  a.nx = pl->nx;
  a.ny = pl->ny;
  a.nz = pl->nz;
  for (int d = 0; d < 3; ++d) {
    a.zeta[d] = static_cast<const T*>(pl->zeta[d]);
    a.ex[d] = static_cast<const T*>(pl->ex[d]);
    a.ec[d] = static_cast<const T*>(pl->ec[d]);
  }
  a.tau = (T)pl->tau;
  a.c2 = (T)pl->opt.c2;
  a.flin = (T)pl->opt.flin;
  a.fcub = (T)pl->opt.fcub;
  a.flog = (T)pl->opt.flog;
}

// Build one pass launch. fields are indices into F (or -1 for a user pointer given later).
// One pass of a split-radix axis (FP32, N = 1024): tiles of P = 2 pencil pairs (4 rows, 5 warps) along x
// and of P = 4 pairs (8 columns: one 32-byte sector per row; 10 warps per transformed field) along strided
// axes where the x extent allows, else 2.
etd_status make_split_launch(etd_plan_s* pl, int op, int axis, const void* in0, const void* in1, void* out0,
                             void* out1, int kind, double fields_rw, Launch& L) {
  const void* fn = find_split_kernel(op);
  if (!fn) return fail(ETD_ERR_UNSUPPORTED, "no split-radix kernel for pass %d", op);
  PassArgs<float> a;
  fill_common<float>(pl, a);
  a.op = op;
  a.axis = axis;
  a.in0 = static_cast<const float*>(in0);
  a.in1 = static_cast<const float*>(in1);
  a.out0 = static_cast<float*>(out0);
  a.out1 = static_cast<float*>(out1);
  a.tw = static_cast<const float*>(pl->stw[axis]);
  a.sn = nullptr;
  a.sc = (float)pl->sc[axis];
  a.lp = SPLIT_LPS;
  int P = 2;
  long long grid = 0;
  if (axis == 0) {
    a.npairs = pl->ny * pl->nz / 2;
    grid = (a.npairs + P - 1) / P;
  } else {
    P = pl->nx % 8 == 0 ? 4 : 2;
    if (pl->nx % (2 * P) != 0) return fail(ETD_ERR_UNSUPPORTED, "x extent %d is not a multiple of 4", pl->nx);
    a.tiles_x = pl->nx / (2 * P);
    grid = (long long)a.tiles_x * ((axis == 1) ? pl->nz : pl->ny);
  }
  a.P = P;
  if (pl->coef) {
    const float* cf = static_cast<const float*>(pl->coef);
    if (op == OP_S1) a.coef = cf + pl->coef_s1;
    else if (op == OP_S2) a.coef = cf + pl->coef_s2;
    else if (op == OP_RK1) a.coef = cf + pl->coef_rk1;
  }
  const int nf = (op == OP_S1 || op == OP_RK1) ? 2 : 1;
  L.fn = fn;
  L.grid = dim3((unsigned)grid);
  L.block = dim3((unsigned)(nf * (P / 2) * 160));
  L.smem = split_smem_bytes(op, P);
  L.kind = kind;
  memcpy(L.args, &a, sizeof(a));
  L.args_size = sizeof(a);
  L.alg_bytes = fields_rw * (double)pl->unknowns * sizeof(float);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
  if (L.smem > (size_t)optin) return fail(ETD_ERR_UNSUPPORTED, "tile needs %zu B of shared memory (max %d)", L.smem, optin);
  if (L.smem > 48 * 1024) {   // the device maximum: one kernel serves launches with different tile sizes
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "cudaFuncSetAttribute(%d B): %s", optin, cudaGetErrorString(e));
  }
  return ETD_OK;
}

template <class T>
etd_status make_launch(etd_plan_s* pl, int op, int axis, const void* in0, const void* in1, void* out0,
                       void* out1, int kind, double fields_rw, Launch& L) {
  if constexpr (sizeof(T) == 4) {
    // split-radix kernels, except under a time-dependent source or boundary data (whose passes add
    // to the reaction field with the odd-extension kernels' epilogues)
    if (pl->split[axis] && !pl->src_on && !pl->bnd_on && op != OP_PACK && op != OP_UNPACK)
      return make_split_launch(pl, op, axis, in0, in1, out0, out1, kind, fields_rw, L);
  }
  const int N = (int)pl->N[axis];
  const KernelInfo* k = find_pass_kernel((int)sizeof(T), N, pl->odd[axis]);
  if (!k) return fail(ETD_ERR_UNSUPPORTED, "no kernel for axis length %d", N);
  PassArgs<T> a;
  fill_common<T>(pl, a);
  a.op = op;
  a.axis = axis;
  a.in0 = static_cast<const T*>(in0);
  a.in1 = static_cast<const T*>(in1);
  a.out0 = static_cast<T*>(out0);
  a.out1 = static_cast<T*>(out1);
  a.tw = static_cast<const T*>(pl->tw[axis]);
  a.sn = static_cast<const T*>(pl->sn[axis]);
  a.sc = (T)pl->sc[axis];
  if (pl->coef && pl->ndim == 2 && axis == 1) {
    const T* cf = static_cast<const T*>(pl->coef);
    if (op == OP_S1 || op == OP_S1S) a.coef = cf + pl->coef_s1;
    else if (op == OP_S2 || op == OP_S2S) a.coef = cf + pl->coef_s2;
    else if (op == OP_RK1 || op == OP_RK1S) a.coef = cf + pl->coef_rk1;
  }
  const bool two = (op == OP_RK1 || op == OP_S1 || op == OP_S2 || op == OP_RK1S || op == OP_S1S || op == OP_S2S);
  const int maxp = 512 / k->tpp > 0 ? 512 / k->tpp : 1;
  int P = 1;
  long long grid = 0;
  if (axis == 0) {
    a.npairs = pl->ny * pl->nz / 2;
    // CTAs of about 64 threads (at least one pencil pair): with many small CTAs per SM the
    // barrier-separated phases of different CTAs interleave (255^3 FP32: P = 8 ran the x passes 13%
    // faster than 512-thread CTAs; 128^3 periodic: 2%).
    P = 64 / k->tpp > 1 ? 64 / k->tpp : 1;
    if (P > maxp) P = maxp;
    while (P > 1 && (a.npairs + P - 1) / P < 2 * pl->num_sms) P /= 2;
    if (P > maxp) P = maxp;
    grid = (a.npairs + P - 1) / P;
  } else {
    const int other = (axis == 1) ? pl->nz : pl->ny;
    // A tile's row segment (2P values) is at least one 32-byte sector: narrower tiles give more CTAs
    // but fetch half-used sectors (at 1023^2 FP32, P = 4 with 128 CTAs ran the y passes 9% faster
    // than P = 2 with 256 CTAs, and P = 1 was 40% slower).
    const int pmin = 16 / (int)sizeof(T);
    const int pmax = 64 / (int)sizeof(T);   // 128-byte row segments: wider tiles gained nothing
    P = maxp < pmax ? maxp : pmax;
    while (P > pmin && (pl->nx / (2 * P)) * (long long)other < 2 * pl->num_sms) P /= 2;
    if (P > maxp) P = maxp;
    while (P > 1 && pl->nx % (2 * P) != 0) P /= 2;
    if (pl->nx % (2 * P) != 0) return fail(ETD_ERR_UNSUPPORTED, "x extent %d not even", pl->nx);
    a.tiles_x = pl->nx / (2 * P);
    grid = (long long)a.tiles_x * other;
  }
  // keep the shared memory of a CTA small enough for the CTAs per SM the kernel was built for
  {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
    const size_t budget = (size_t)optin / (size_t)k->min_blocks - 2048;
    while (P > 1 && pass_smem_bytes(*k, P, two ? 2 : 1) > budget) {
      P /= 2;
      if (axis == 0) grid = (a.npairs + P - 1) / P;
    }
    if (axis != 0) {
      a.tiles_x = pl->nx / (2 * P);
      grid = (long long)a.tiles_x * ((axis == 1) ? pl->nz : pl->ny);
    }
  }
  a.P = P;
  a.lp = pair_stride(*k, P);
  L.fn = (op >= 0 && op < OP_COUNT && k->fn_op[op]) ? k->fn_op[op] : k->fn;
  L.grid = dim3((unsigned)grid);
  L.block = dim3((unsigned)(P * k->tpp));
  L.smem = pass_smem_bytes(*k, P, two ? 2 : 1);
  L.kind = kind;
  // One kernel serves every axis of a given length, with different tile sizes, so the opt-in
  // limit is raised to the device maximum (not to this launch's size, which a later launch of the
  // same kernel could then undercut).
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
  // Weight tables of FP32 2D plans: kernels of axis lengths up to 1536 stage their tile's rows in shared
  // memory before the dependency wait (in place of the zeta table, which the table epilogue does not
  // read); a launch whose rows do not fit, or are not whole 16-byte chunks, gets no tables and evaluates
  // the weights per mode. Longer axes read the tables from global memory.
  if constexpr (sizeof(T) == 4) {
    if (a.coef && two && k->min_blocks == 1 && k->N <= 1536) {
      const int fpm = (op == OP_S1 || op == OP_S1S) ? 2 : 1;
      const size_t need = L.smem - (size_t)N * sizeof(float) + 16 + (size_t)N * 2 * P * fpm * sizeof(float);
      if ((2 * P * fpm) % 4 == 0 && need <= (size_t)optin) {
        a.coef_smem = 1;
        L.smem = need;
      } else {
        a.coef = nullptr;
      }
    }
  }
  memcpy(L.args, &a, sizeof(a));
  L.args_size = sizeof(a);
  L.alg_bytes = fields_rw * (double)pl->unknowns * sizeof(T);
  if (L.smem > (size_t)optin) return fail(ETD_ERR_UNSUPPORTED, "tile needs %zu B of shared memory (max %d)", L.smem, optin);
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "cudaFuncSetAttribute(%d B): %s", optin, cudaGetErrorString(e));
  }
  return ETD_OK;
}

// Pass kernels are launched with programmatic stream serialization (PDL): the next pass may be
// scheduled while the previous one drains, and waits in-kernel (griddepcontrol.wait) before reading
// its inputs. ETD_PDL=0 disables it.
etd_status launch(const Launch& L, cudaStream_t s) {
  static const int use_pdl = env_int("ETD_PDL", 1);
  void* argv[1] = {const_cast<unsigned char*>(L.args)};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = L.grid;
  cfg.blockDim = L.block;
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = use_pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelExC(&cfg, L.fn, argv);
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return ETD_OK;
}

// Sets the source fields of the step's launches: the reaction passes (stage 1 at t_n, stage 2 at
// t_n + c2 tau) read the step count and start time; the last pass of a step advances the count.
template <class T>
void apply_source(etd_plan_s* pl) {
  if (!pl->src_on || pl->step.empty()) return;
  const T* tab = static_cast<const T*>(pl->src_tab);
  int nreact = 0;
  for (Launch& L : pl->step) {
    if (L.kind == PK_BOUNDARY) continue;   // boundary-data launches (their transforms are not REACT)
    PassArgs<T>* a = reinterpret_cast<PassArgs<T>*>(L.args);
    if (a->op != OP_REACT) continue;
    a->src_gx = tab;
    a->src_gy = tab + pl->nx;
    a->src_gz = pl->ndim == 3 ? tab + pl->nx + pl->ny : nullptr;
    a->step_ctr = static_cast<const unsigned long long*>(pl->clock);
    a->src_t0 = reinterpret_cast<const double*>(static_cast<const char*>(pl->clock) + 8);
    a->src_amp = pl->src_amp;
    a->src_rate = pl->src_rate;
    a->src_c = nreact++ == 0 ? 0.0 : pl->opt.c2;
  }
  reinterpret_cast<PassArgs<T>*>(pl->step.back().args)->step_inc = static_cast<unsigned long long*>(pl->clock);
}

__global__ void source_clock_kernel(unsigned long long* steps, double* t0p, double t0) {
  *steps = 0;
  *t0p = t0;
}

// A launch of one of the boundary-data kernels (boundary.cuh) on the plan's B field.
template <class T>
Launch bnd_launch(const etd_plan_s* pl, const void* fn, const BndArgs<T>& a, double fields_rw) {
  static_assert(sizeof(BndArgs<T>) <= sizeof(Launch::args), "launch argument buffer too small");
  Launch L;
  L.fn = fn;
  const long long blocks = (a.n + 255) / 256;
  L.grid = dim3((unsigned)(blocks < 4LL * pl->num_sms ? blocks : 4LL * pl->num_sms));
  L.block = dim3(256);
  L.smem = 0;
  L.kind = PK_BOUNDARY;
  memcpy(L.args, &a, sizeof(a));
  L.args_size = sizeof(a);
  L.alg_bytes = fields_rw * (double)pl->nfield * sizeof(T);
  return L;
}

// Appends the launches that add M_II^{-1} b(t_stage) to the reaction field `target` (pitched, spectral
// along every axis but the last): BUILD, DST along every axis, SCALE, DST along the last axis, ADD.
template <class T>
etd_status append_boundary(etd_plan_s* pl, int stage, void* target, std::vector<Launch>& out) {
  BndArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.ndim = pl->ndim;
  a.nx = pl->nx;
  a.ny = pl->ny;
  a.nz = pl->nz;
  a.n = (long long)pl->nfield;
  T* B = static_cast<T*>(pl->bnd_field);
  a.out = B;
  a.g = pl->bnd_dev + (size_t)stage * 2 * pl->bnd_count;
  a.count = pl->bnd_count;
  const long long Nx = pl->nx, Ny = pl->ny, Nz = pl->nz;
  if (pl->ndim == 3) {
    const long long fx = (Nz + 1) * (Ny + 1), fy = (Nz + 1) * (Nx + 1), fz = (Ny + 1) * (Nx + 1);
    const long long sz[6] = {fx, fx, fy, fy, fz, fz};
    for (int f = 1; f < 6; ++f) a.off[f] = a.off[f - 1] + sz[f - 1];
  } else {
    const long long sz[4] = {Ny + 1, Ny + 1, Nx + 1, Nx + 1};
    for (int f = 1; f < 4; ++f) a.off[f] = a.off[f - 1] + sz[f - 1];
  }
  for (int d = 0; d < 3; ++d) a.h[d] = d < pl->ndim ? pl->h[d] : 1.0;
  a.D = pl->D;
  a.flin = pl->opt.flin;
  a.fcub = pl->opt.fcub;
  a.ia[0] = pl->bnd_ia;
  a.ia[1] = pl->bnd_ia + Nx;
  a.ia[2] = pl->bnd_ia + Nx + Ny;
  out.push_back(bnd_launch<T>(pl, reinterpret_cast<const void*>(&bnd_build_kernel<T>), a, 1));
  Launch L;
  etd_status st;
  for (int ax = 0; ax <= pl->ndim; ++ax) {   // every axis, then the last axis again after SCALE
    const int axis = ax < pl->ndim ? ax : pl->ndim - 1;
    if (ax == pl->ndim) out.push_back(bnd_launch<T>(pl, reinterpret_cast<const void*>(&bnd_scale_kernel<T>), a, 2));
    if ((st = make_launch<T>(pl, OP_TRANSFORM, axis, B, nullptr, B, nullptr, PK_BOUNDARY, 2, L)) != ETD_OK) return st;
    out.push_back(L);
  }
  a.out = static_cast<T*>(target);
  a.in = B;
  out.push_back(bnd_launch<T>(pl, reinterpret_cast<const void*>(&bnd_add_kernel<T>), a, 3));
  return ETD_OK;
}

template <class T>
etd_status build_step(etd_plan_s* pl) {
  void** F = pl->F;
  enum { V = 0, N0 = 1, V2 = 2, PF = 3, N2 = 4, VS = 5 };
  pl->step.clear();
  Launch L;
  etd_status st;
  // The stage passes of the last axis: on plans that keep V~ (V transformed along the last axis, written
  // by the step's last pass) they read it instead of transforming V, one DST fewer per step for one more
  // field written.
  const bool sp = pl->spec;
  const int op_s1 = sp ? OP_S1S : OP_S1, op_s2 = sp ? OP_S2S : OP_S2, op_rk1 = sp ? OP_RK1S : OP_RK1;
  void* const s1_in = sp ? F[VS] : F[V];
  void* const s2_out1 = sp ? F[VS] : nullptr;
  const double s2_rw = sp ? 4 : 3;
#define ADD(op, axis, i0, i1, o0, o1, kind, rw)                                               \
  do {                                                                                         \
    st = make_launch<T>(pl, op, axis, i0, i1, o0, o1, kind, rw, L);                            \
    if (st != ETD_OK) return st;                                                               \
    pl->step.push_back(L);                                                                     \
  } while (0)
  // nonhomogeneous Dirichlet data: the stage's reaction field receives M_II^{-1} b(t_stage)
#define BND(stage, field)                                                                      \
  do {                                                                                         \
    if (pl->bnd_on && (st = append_boundary<T>(pl, stage, field, pl->step)) != ETD_OK) return st; \
  } while (0)
  if (pl->ndim == 2) {
    if (pl->scheme == 2) {
      ADD(OP_REACT, 0, F[V], nullptr, F[N0], nullptr, PK_REACT, 2);
      BND(0, F[N0]);
      ADD(op_s1, 1, s1_in, F[N0], F[V2], F[PF], PK_S1, 4);
      ADD(OP_REACT, 0, F[V2], nullptr, F[N2], nullptr, PK_REACT, 2);
      BND(1, F[N2]);
      ADD(op_s2, 1, F[N2], F[PF], F[V], s2_out1, PK_S2, s2_rw);
    } else {
      ADD(OP_REACT, 0, F[V], nullptr, F[N0], nullptr, PK_REACT, 2);
      BND(0, F[N0]);
      ADD(op_rk1, 1, s1_in, F[N0], F[V], s2_out1, PK_RK1, s2_rw);
    }
  } else {
    ADD(OP_TRANSFORM, 1, F[V], nullptr, F[V2], nullptr, PK_TRANSFORM, 2);
    ADD(OP_REACT, 0, F[V2], nullptr, F[N0], nullptr, PK_REACT, 2);
    ADD(OP_TRANSFORM, 1, F[N0], nullptr, F[N0], nullptr, PK_TRANSFORM, 2);
    BND(0, F[N0]);
    if (pl->scheme == 2) {
      ADD(op_s1, 2, s1_in, F[N0], F[V2], F[PF], PK_S1, 4);
      ADD(OP_TRANSFORM, 1, F[V2], nullptr, F[V2], nullptr, PK_TRANSFORM, 2);
      ADD(OP_REACT, 0, F[V2], nullptr, F[N2], nullptr, PK_REACT, 2);
      ADD(OP_TRANSFORM, 1, F[N2], nullptr, F[N2], nullptr, PK_TRANSFORM, 2);
      BND(1, F[N2]);
      ADD(op_s2, 2, F[N2], F[PF], F[V], s2_out1, PK_S2, s2_rw);
    } else {
      ADD(op_rk1, 2, s1_in, F[N0], F[V], s2_out1, PK_RK1, s2_rw);
    }
  }
#undef BND
#undef ADD
  return ETD_OK;
}

// entry: dense u -> state; exit: state -> dense u
template <class T>
etd_status entry_exit(etd_plan_s* pl, bool entry, void* u, std::vector<Launch>& out) {
  Launch L;
  etd_status st;
  void** F = pl->F;
  out.clear();
  if (entry) {
    st = make_launch<T>(pl, OP_ENTRY, 0, u, nullptr, F[0], nullptr, PK_ENTRY_EXIT, 2, L);
    if (st != ETD_OK) return st;
    out.push_back(L);
    if (pl->ndim == 3) {
      st = make_launch<T>(pl, OP_TRANSFORM, 1, F[0], nullptr, F[0], nullptr, PK_ENTRY_EXIT, 2, L);
      if (st != ETD_OK) return st;
      out.push_back(L);
    }
    if (pl->spec) {   // V~ for the first step's stage pass
      st = make_launch<T>(pl, OP_TRANSFORM, pl->ndim - 1, F[0], nullptr, F[5], nullptr, PK_ENTRY_EXIT, 2, L);
      if (st != ETD_OK) return st;
      out.push_back(L);
    }
  } else {
    if (pl->ndim == 3) {
      st = make_launch<T>(pl, OP_TRANSFORM, 1, F[0], nullptr, F[2], nullptr, PK_ENTRY_EXIT, 2, L);
      if (st != ETD_OK) return st;
      out.push_back(L);
      st = make_launch<T>(pl, OP_EXIT, 0, F[2], nullptr, u, nullptr, PK_ENTRY_EXIT, 2, L);
    } else {
      st = make_launch<T>(pl, OP_EXIT, 0, F[0], nullptr, u, nullptr, PK_ENTRY_EXIT, 2, L);
    }
    if (st != ETD_OK) return st;
    out.push_back(L);
  }
  return ETD_OK;
}

// ---------------------------------------------------------------------------------------------
// Tensor-core transform passes (GEMM routes).

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link to libcuda).
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map of a row-major matrix of rows x cols elements of `elem` bytes, tile box {box_cols, box_rows}.
etd_status make_tmap(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int elem, uint64_t cols, uint64_t rows,
                     uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(ETD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (cols * (uint64_t)elem) % 16)
    return fail(ETD_ERR_UNSUPPORTED, "tensor map: base or row pitch not 16-byte aligned");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * (cuuint64_t)elem};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ETD_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return ETD_OK;
}

// Round to TF32 (10 stored mantissa bits), to nearest, ties to even; |v| <= 1 here.
float round_tf32(double v) {
  float f = (float)v;
  uint32_t b;
  memcpy(&b, &f, 4);
  b += 0xFFFu + ((b >> 13) & 1u);
  b &= 0xFFFFE000u;
  memcpy(&f, &b, 4);
  return f;
}
// Round to bfloat16, to nearest, ties to even; returns the bits and the rounded value.
uint16_t round_bf16(double v, double* back) {
  float f = (float)v;
  uint32_t b;
  memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  const uint16_t h = (uint16_t)(b >> 16);
  const uint32_t w = (uint32_t)h << 16;
  float r;
  memcpy(&r, &w, 4);
  *back = (double)r;
  return h;
}

// S_a[j][k] = sqrt(2/N) sin(pi (j k mod 2N) / N) (periodic: N^{-1/2} cas(2 pi (j k mod N) / N)), j, k < N,
// in FP64, stored per axis in the operand
// format of the route: fp32 rounded to TF32, or bf16 hi = rn(S), lo = rn(S - hi).
etd_status upload_gemm_tables(etd_plan_s* pl) {
  size_t offs[3][2], total = 0;
  const bool split = pl->gemm - 1 == GR_BF16X3;
  for (int a = 0; a < pl->ndim; ++a) {
    const size_t n2 = (size_t)pl->N[a] * pl->N[a];
    for (int part = 0; part < (split ? 2 : 1); ++part) {
      offs[a][part] = total;
      total += ((n2 * (split ? 2 : 4)) + 255) & ~(size_t)255;
    }
  }
  std::vector<unsigned char> h(total, 0);
  for (int a = 0; a < pl->ndim; ++a) {
    const long long n = pl->N[a];
    const double s0 = pl->periodic ? 1.0 / sqrt((double)n) : sqrt(2.0 / (double)n);
    for (long long j = 0; j < n; ++j)
      for (long long k = 0; k < n; ++k) {
        double v;
        if (pl->periodic) {   // Hartley: cas(2 pi j k / n), j k reduced mod n
          const double t = 2.0 * M_PI * (double)((j * k) % n) / (double)n;
          v = s0 * (cos(t) + sin(t));
        } else {
          v = s0 * sin(M_PI * (double)((j * k) % (2 * n)) / (double)n);
        }
        const size_t e = (size_t)(j * n + k);
        if (!split) {
          const float f = round_tf32(v);
          memcpy(&h[offs[a][0] + 4 * e], &f, 4);
        } else {
          double hv, lv;
          const uint16_t hb = round_bf16(v, &hv);
          const uint16_t lb = round_bf16(v - hv, &lv);
          memcpy(&h[offs[a][0] + 2 * e], &hb, 2);
          memcpy(&h[offs[a][1] + 2 * e], &lb, 2);
        }
      }
  }
  ETD_CUDA(cudaMalloc(&pl->gtab, total));
  ETD_CUDA(cudaMemcpy(pl->gtab, h.data(), total, cudaMemcpyHostToDevice));
  for (int a = 0; a < pl->ndim; ++a) {
    pl->gS[a][0] = static_cast<char*>(pl->gtab) + offs[a][0];
    pl->gS[a][1] = split ? static_cast<char*>(pl->gtab) + offs[a][1] : nullptr;
  }
  ETD_CUDA(cudaMalloc(&pl->dev_err, sizeof(int)));
  ETD_CUDA(cudaMemset(pl->dev_err, 0, sizeof(int)));
  for (int route = 0; route < 2; ++route)
    for (int bn = 32; bn <= 256; bn *= 2) {
      const GemmKernelInfo* k = find_gemm_kernel(bn, route);
      if (!k) return fail(ETD_ERR_UNSUPPORTED, "no tensor-core pass for tile width %d", bn);
      ETD_CUDA(cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k->smem));
    }
  return ETD_OK;
}

// One tensor-core pass contracting paper axis a of field `in` (pitched, axis a contiguous):
// out0[k * R + r] = epi((in S_a)[r][k]).
etd_status make_gemm_launch(etd_plan_s* pl, int a, const void* in, const void* in1, void* out0, void* out1, int op,
                            int kind, double fields_rw, Launch& L, bool stall = false) {
  const int K = (int)pl->N[a];
  const int R = (int)(pl->nfield / (size_t)K);
  const int route = pl->gemm - 1;
  const int mt = (R + 127) / 128;
  // widest tile that still gives every SM a CTA (wider tiles re-read the field fewer times)
  int bn = 256;
  while (bn > K) bn /= 2;
  while (bn > 64 && (long long)mt * ((K + bn - 1) / bn) < pl->num_sms) bn /= 2;
  if (bn > K) bn = 32;
  const GemmKernelInfo* k = find_gemm_kernel(bn, route);
  if (!k) return fail(ETD_ERR_UNSUPPORTED, "no tensor-core pass for tile width %d", bn);
  const int nt = (K + bn - 1) / bn;
  GemmParams prm;
  memset(&prm, 0, sizeof(prm));
  etd_status st = make_tmap(&prm.ta, in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)K, (uint64_t)R, 32, 128,
                            CU_TENSOR_MAP_SWIZZLE_128B);
  if (st != ETD_OK) return st;
  if (route == GR_TF32) {
    st = make_tmap(&prm.tb0, pl->gS[a][0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)K, (uint64_t)K, 32,
                   (uint32_t)bn, CU_TENSOR_MAP_SWIZZLE_128B);
  } else {
    st = make_tmap(&prm.tb0, pl->gS[a][0], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)K, (uint64_t)K, 32,
                   (uint32_t)bn, CU_TENSOR_MAP_SWIZZLE_64B);
    if (st == ETD_OK)
      st = make_tmap(&prm.tb1, pl->gS[a][1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)K, (uint64_t)K, 32,
                     (uint32_t)bn, CU_TENSOR_MAP_SWIZZLE_64B);
  }
  if (st != ETD_OK) return st;
  GemmArgs& g = prm.g;
  g.op = op;
  g.R = R;
  g.K = K;
  g.row_split = pl->ndim == 3 ? pl->nx : 0;
  g.in1 = static_cast<const float*>(in1);
  g.out0 = static_cast<float*>(out0);
  g.out1 = static_cast<float*>(out1);
  const int last = pl->ndim - 1;   // spectral passes contract the last axis; rows are (y,) x
  g.zx = static_cast<const float*>(pl->zeta[0]);
  g.ex = static_cast<const float*>(pl->ex[0]);
  g.cx = static_cast<const float*>(pl->ec[0]);
  g.zy = static_cast<const float*>(pl->zeta[1]);
  g.ey = static_cast<const float*>(pl->ex[1]);
  g.cy = static_cast<const float*>(pl->ec[1]);
  g.zk = static_cast<const float*>(pl->zeta[last]);
  g.ek = static_cast<const float*>(pl->ex[last]);
  g.ck = static_cast<const float*>(pl->ec[last]);
  g.tau = (float)pl->tau;
  g.c2 = (float)pl->opt.c2;
  g.flin = (float)pl->opt.flin;
  g.fcub = (float)pl->opt.fcub;
  g.flog = (float)pl->opt.flog;
  g.err = pl->dev_err;
  g.stall = stall ? 1 : 0;
  L.fn = k->fn;
  L.grid = dim3((unsigned)(mt * nt));
  L.block = dim3((unsigned)k->threads);
  L.smem = k->smem;
  L.kind = kind;
  memcpy(L.args, &prm, sizeof(prm));
  L.args_size = sizeof(prm);
  L.alg_bytes = fields_rw * (double)pl->unknowns * 4.0;
  return ETD_OK;
}

// Time step of the GEMM routes: per stage d inverse passes (the d-th applies the reaction) and d
// forward passes (the last applies the ETD combination), alternating between two scratch fields.
etd_status build_step_gemm(etd_plan_s* pl) {
  void** F = pl->F;
  enum { V = 0, T1 = 1, V2 = 2, PF = 3, T2 = 4 };
  const int d = pl->ndim;
  pl->step.clear();
  auto stage = [&](int in, int last_op, int out0, int in1, int out1, int kind_last, double rw_last) -> etd_status {
    int cur = in;
    for (int p = 0; p < 2 * d; ++p) {
      const bool last = p == 2 * d - 1;
      const int dst = last ? out0 : (p % 2 == 0 ? T1 : T2);
      const int op = last ? last_op : (p == d - 1 ? GE_REACT : GE_PLAIN);
      const int kind = last ? kind_last : (p == d - 1 ? PK_REACT : PK_TRANSFORM);
      Launch L;
      etd_status st = make_gemm_launch(pl, p % d, F[cur], last ? F[in1] : nullptr, F[dst],
                                       (last && out1 >= 0) ? F[out1] : nullptr, op, kind, last ? rw_last : 2.0, L);
      if (st != ETD_OK) return st;
      pl->step.push_back(L);
      cur = dst;
    }
    return ETD_OK;
  };
  etd_status st;
  if (pl->scheme == 2) {
    if ((st = stage(V, GE_S1, V2, V, PF, PK_S1, 4.0)) != ETD_OK) return st;
    if ((st = stage(V2, GE_S2, V, PF, -1, PK_S2, 3.0)) != ETD_OK) return st;
  } else {
    if ((st = stage(V, GE_RK1, V, V, -1, PK_RK1, 3.0)) != ETD_OK) return st;
  }
  return ETD_OK;
}

// GEMM routes: entry packs the dense field into V and applies d forward passes (back to the
// [z][y][x] layout); exit applies d passes into scratch and unpacks.
etd_status entry_exit_gemm(etd_plan_s* pl, bool entry, void* u, std::vector<Launch>& out) {
  void** F = pl->F;
  enum { V = 0, T1 = 1, T2 = 4 };
  const int d = pl->ndim;
  Launch L;
  etd_status st;
  out.clear();
  if (entry) {
    if ((st = make_launch<float>(pl, OP_PACK, 0, u, nullptr, F[V], nullptr, PK_ENTRY_EXIT, 2, L)) != ETD_OK) return st;
    out.push_back(L);
  }
  int cur = V;
  for (int p = 0; p < d; ++p) {
    const int dst = (entry && p == d - 1) ? V : (p % 2 == 0 ? T1 : T2);
    const bool stall = entry && p == 0 && pl->opt.debug == ETD_DEBUG_STALL_FIRST_GEMM_PASS;
    if ((st = make_gemm_launch(pl, p, F[cur], nullptr, F[dst], nullptr, GE_PLAIN, PK_ENTRY_EXIT, 2.0, L, stall)) !=
        ETD_OK)
      return st;
    out.push_back(L);
    cur = dst;
  }
  if (!entry) {
    if ((st = make_launch<float>(pl, OP_UNPACK, 0, F[cur], nullptr, u, nullptr, PK_ENTRY_EXIT, 2, L)) != ETD_OK)
      return st;
    out.push_back(L);
  }
  return ETD_OK;
}

// Reads (and clears) the error word of the tensor-core passes; call after synchronising.
etd_status check_dev_err(etd_plan_s* pl) {
  if (!pl->dev_err) return ETD_OK;
  int h = 0;
  ETD_CUDA(cudaMemcpy(&h, pl->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    ETD_CUDA(cudaMemset(pl->dev_err, 0, sizeof(int)));
    return fail(ETD_ERR_TIMEOUT, "a tensor-core pass gave up waiting for its pipeline; the field is invalid");
  }
  return ETD_OK;
}

etd_status entry_exit_any(etd_plan_s* pl, bool entry, void* u, std::vector<Launch>& out) {
  if (pl->gemm) return entry_exit_gemm(pl, entry, u, out);
  return pl->elem == 4 ? entry_exit<float>(pl, entry, u, out) : entry_exit<double>(pl, entry, u, out);
}

// FP64 on the host, rounded once to T, appended to h for one axis of length n: the per-pass twiddle
// tables (pass with NS > 1 and radix R holds exp(2 pi i k r / (NS R)) at [(r-1)*NS + k], k < NS,
// r = 1..R-1, the layout the Stockham passes read), sin(pi j / n), and per mode i the values
// zeta = tau D mu_i, exp(-zeta), exp(-c2 zeta) with mu_i = (6/h^2)(1 - cos)/(2 + cos) of theta = i pi / n
// (periodic axes: theta = 2 pi i / n, mode 0 included with zeta = 0).
// offs receives the five table starts (element offsets into h).
template <class T>
void append_axis_tables(const KernelInfo* k, int n, double hh, double tauD, double c2, std::vector<T>& h,
                        size_t offs[5], bool periodic = false) {
  offs[0] = h.size();
  int NS = 1;
  size_t t = 0;
  for (int i = 0; i < 4 && k->radix[i]; ++i) {
    const int R = k->radix[i];
    if (NS > 1) {
      for (int r = 1; r < R; ++r)
        for (int kk = 0; kk < NS; ++kk, ++t) {
          const long long num = (long long)kk * r % ((long long)NS * R);
          const double ang = 2.0 * M_PI * (double)num / (double)(NS * R);
          h.push_back((T)cos(ang));
          h.push_back((T)sin(ang));
        }
    }
    NS *= R;
  }
  if (t == 0) {
    h.push_back(T(1));
    h.push_back(T(0));
  }
  offs[1] = h.size();
  for (int j = 0; j < n; ++j) h.push_back((T)sin(M_PI * (double)j / (double)n));
  offs[2] = h.size();
  offs[3] = offs[2] + n;
  offs[4] = offs[2] + 2 * (size_t)n;
  h.resize(h.size() + 3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double zeta = 0.0;
    if (i > 0) {
      const double th = (periodic ? 2.0 * M_PI : M_PI) * (double)i / (double)n;
      const double s = sin(0.5 * th);
      const double mu = 12.0 / (hh * hh) * s * s / (2.0 + cos(th));  // (6/h^2)(1-cos)/(2+cos)
      zeta = tauD * mu;
    }
    h[offs[2] + i] = (T)zeta;
    h[offs[3] + i] = (T)exp(-zeta);
    h[offs[4] + i] = (T)exp(-c2 * zeta);
  }
}

// Twiddle table of a split-radix axis (split_dst.cuh), FP64 values rounded once, appended at a 16-byte
// boundary: the pre-twiddles (1/2) sqrt(2/N) e^{i pi k/N} (k < 512) and (1/2) sqrt(2/N) e^{i pi k/(N/2)}
// (k < 256) of the two DST-III stages, and e^{2 pi i n k/512}, e^{2 pi i n k/256} for the twiddle step
// of the 512- and 256-point FFTs.
template <class T>
size_t append_split_tables(std::vector<T>& h) {
  while (h.size() % 4) h.push_back(T(0));
  const size_t off = h.size();
  const double n = (double)SPLIT_N, s = 0.5 * sqrt(2.0 / n);
  auto put = [&](double ang, double scale) {
    h.push_back((T)(scale * cos(ang)));
    h.push_back((T)(scale * sin(ang)));
  };
  for (int k = 0; k < 512; ++k) put(M_PI * k / n, s);
  for (int m = 1; m < 16; ++m)
    for (int k = 0; k < 32; ++k) put(2.0 * M_PI * (double)(m * k) / 512.0, 1.0);
  for (int k = 0; k < 256; ++k) put(M_PI * k / (0.5 * n), s);
  for (int m = 1; m < 16; ++m)
    for (int k = 0; k < 16; ++k) put(2.0 * M_PI * (double)(m * k) / 256.0, 1.0);
  return off;
}

// phi_1(z), phi_2(z) in FP64 for z <= 0 (Section 2.2): the Taylor series sum_m z^m/(m+k)! for |z| < 1/2
// (24 terms, truncation below 1e-20), the closed forms (e^z - 1)/z and (e^z - 1 - z)/z^2 through expm1
// above, where their cancellation costs at most a few ulps.
void phi12_fp64(double z, double& p1, double& p2) {
  if (fabs(z) < 0.5) {
    double s1 = 0, s2 = 0, t = 1, f1 = 1, f2 = 0.5;
    for (int m = 0; m < 24; ++m) {
      s1 += t * f1;
      s2 += t * f2;
      t *= z;
      f1 /= (m + 2);
      f2 /= (m + 3);
    }
    p1 = s1;
    p2 = s2;
  } else {
    const double e = expm1(z);
    p1 = e / z;
    p2 = (e - z) / (z * z);
  }
}

// Per-mode phi-function weights of a 2D FP32 plan (FFT routes, both the default and the split-radix
// kernels read them), computed in FP64 from zeta = tau D (mu_x + mu_y) with the closed-form 1D rates (those of append_axis_tables) and
// rounded once to FP32; layouts as documented for PassArgs::coef (the exponentials e^{-z}, e^{-c2 z} are
// products of the per-axis tables).
template <class T>
etd_status upload_coef_tables(etd_plan_s* pl) {
  const int nx = pl->nx, ny = pl->ny;
  const size_t modes = (size_t)nx * ny;
  const double tauD = pl->tau * pl->D, c2 = pl->opt.c2, tau = pl->tau;
  std::vector<double> mx(nx), my(ny);
  auto mu = [](int i, int n, double hh) {
    if (i == 0) return 0.0;
    const double th = M_PI * (double)i / (double)n, s = sin(0.5 * th);
    return 12.0 / (hh * hh) * s * s / (2.0 + cos(th));   // (6/h^2)(1 - cos)/(2 + cos)
  };
  for (int i = 0; i < nx; ++i) mx[i] = mu(i, nx, pl->h[0]);
  for (int j = 0; j < ny; ++j) my[j] = mu(j, ny, pl->h[1]);
  std::vector<T> h;
  if (pl->scheme == 2) {
    pl->coef_s1 = 0;
    pl->coef_s2 = 2 * modes;
    h.resize(3 * modes);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t m = (size_t)j * nx + i;
        const double z = tauD * (mx[i] + my[j]);
        double p1, p2, p1c, p2c;
        phi12_fp64(-z, p1, p2);
        phi12_fp64(-c2 * z, p1c, p2c);
        h[2 * m + 0] = (T)(c2 * tau * p1c);
        h[2 * m + 1] = (T)(tau * (p1 - p2 / c2));
        h[2 * modes + m] = (T)(tau * p2 / c2);
      }
  } else {
    pl->coef_rk1 = 0;
    h.resize(modes);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t m = (size_t)j * nx + i;
        double p1, p2;
        phi12_fp64(-tauD * (mx[i] + my[j]), p1, p2);
        h[m] = (T)(tau * p1);
      }
  }
  ETD_CUDA(cudaMalloc(&pl->coef, h.size() * sizeof(T)));
  ETD_CUDA(cudaMemcpy(pl->coef, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ETD_OK;
}

template <class T>
etd_status upload_tables(etd_plan_s* pl) {
  std::vector<T> h;
  size_t offs[3][5], soff[3] = {0, 0, 0};
  for (int a = 0; a < pl->ndim; ++a) {
    const KernelInfo* k = find_pass_kernel((int)sizeof(T), (int)pl->N[a], pl->odd[a]);
    if (!k) return fail(ETD_ERR_UNSUPPORTED, "no kernel for axis length %lld", (long long)pl->N[a]);
    append_axis_tables<T>(k, (int)pl->N[a], pl->h[a], pl->tau * pl->D, pl->opt.c2, h, offs[a], pl->periodic != 0);
    if (pl->split[a]) soff[a] = append_split_tables<T>(h);
    pl->sc[a] = pl->periodic ? 0.5 / sqrt((double)pl->N[a]) : 0.5 * sqrt(2.0 / (double)pl->N[a]);
  }
  ETD_CUDA(cudaMalloc(&pl->tables, h.size() * sizeof(T)));
  ETD_CUDA(cudaMemcpy(pl->tables, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  T* base = static_cast<T*>(pl->tables);
  for (int a = 0; a < pl->ndim; ++a) {
    pl->tw[a] = base + offs[a][0];
    pl->sn[a] = base + offs[a][1];
    pl->zeta[a] = base + offs[a][2];
    pl->ex[a] = base + offs[a][3];
    pl->ec[a] = base + offs[a][4];
    pl->stw[a] = pl->split[a] ? base + soff[a] : nullptr;
  }
  for (int a = pl->ndim; a < 3; ++a) {   // unused third axis in 2D: point at axis 0 (never read)
    pl->tw[a] = pl->tw[0];
    pl->sn[a] = pl->sn[0];
    pl->zeta[a] = pl->zeta[0];
    pl->ex[a] = pl->ex[0];
    pl->ec[a] = pl->ec[0];
  }
  return ETD_OK;
}

etd_status destroy_graph(etd_plan_s* pl) {
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  pl->graph = nullptr;
  pl->graph_steps = 0;
  return ETD_OK;
}

etd_status ensure_graph(etd_plan_s* pl, int gsteps) {
  if (pl->graph && pl->graph_steps == gsteps) return ETD_OK;
  destroy_graph(pl);
  if (!pl->cap_stream) ETD_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  ETD_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
  etd_status st = ETD_OK;
  for (int s = 0; s < gsteps && st == ETD_OK; ++s)
    for (const Launch& L : pl->step)
      if ((st = launch(L, pl->cap_stream)) != ETD_OK) break;
  cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  if (st != ETD_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&pl->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  pl->graph_steps = gsteps;
  return ETD_OK;
}

// Runs with nonhomogeneous Dirichlet data: per time step the callback fills the pinned staging
// buffer for each stage time, one copy moves it to the device, the step's launches follow, and the
// stream is synchronised before the buffer is refilled.
etd_status run_steps_boundary(etd_plan_s* pl, int64_t nsteps, double t0, cudaStream_t s) {
  const int stages = pl->scheme == 2 ? 2 : 1;
  const size_t per = 2 * (size_t)pl->bnd_count;
  for (int64_t n = 0; n < nsteps; ++n) {
    const double tn = t0 + (double)n * pl->tau;
    for (int k = 0; k < stages; ++k) {
      const double t = tn + (k ? pl->opt.c2 * pl->tau : 0.0);
      double* hb = pl->bnd_host + k * per;
      const int rc = pl->bnd_fn(t, hb, hb + pl->bnd_count, pl->bnd_ctx);
      if (rc != 0) return fail(ETD_ERR_INVALID_ARG, "boundary callback returned %d at t = %g", rc, t);
    }
    ETD_CUDA(cudaMemcpyAsync(pl->bnd_dev, pl->bnd_host, stages * per * sizeof(double), cudaMemcpyHostToDevice, s));
    for (const Launch& L : pl->step) {
      etd_status st = launch(L, s);
      if (st != ETD_OK) return st;
    }
    ETD_CUDA(cudaStreamSynchronize(s));
  }
  return ETD_OK;
}

etd_status run_steps(etd_plan_s* pl, int64_t nsteps, cudaStream_t s) {
  const int G = env_int("ETD_GRAPH_STEPS", 32);
  int64_t done = 0;
  if (G > 0 && nsteps >= G) {
    etd_status st = ensure_graph(pl, G);
    if (st != ETD_OK) return st;
    for (; done + G <= nsteps; done += G) ETD_CUDA(cudaGraphLaunch(pl->graph, s));
  }
  for (; done < nsteps; ++done)
    for (const Launch& L : pl->step) {
      etd_status st = launch(L, s);
      if (st != ETD_OK) return st;
    }
  return ETD_OK;
}

// ---------------------------------------------------------------------------------------------
// Batches of independent 2D problems (uneven meshes and diffusion coefficients, common tau).
// A pass of the time step is launched once per distinct length of the transformed axis: the launch
// covers every tile of every problem with that length, each CTA reading its problem's descriptor.
// The tile size of each launch is picked at creation by timing the candidates on the workspace.

struct BatchGroup {
  const void* fn = nullptr;     // pass_kernel_batched<T, N, ODD>
  int axis = 0, op = 0, N = 0, P = 1, nbuf = 1, kind = 0;
  int pass = 0;                 // index of the pass in the time step (groups of one pass are independent)
  size_t smem = 0;
  int nctas = 0, tpp = 1;
  std::vector<int> inst;        // problems in this group
  void* d_descs = nullptr;      // PassArgs<T>[inst.size()]
  void* d_map = nullptr;        // int2[nctas]
  double alg_bytes = 0;
};

}  // namespace

struct etd_batch_s {
  int count = 0, elem = 4, scheme = 2;
  int periodic = 0;                // every problem periodic (Hartley kernels), else homogeneous Dirichlet
  etd_options opt{};
  double tau = 0;
  int device = 0, num_sms = 148, optin = 0;
  std::vector<int> nx, ny, oddx, oddy;
  std::vector<double> hx, hy, Dv;
  std::vector<size_t> field_off;   // element offset of problem i's five fields
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* tables = nullptr;
  void* d_user = nullptr;          // T*[count], the caller's fields of the current run
  void* d_aux = nullptr;           // descriptors and tile maps of all groups
  size_t aux_bytes = 0;
  std::vector<BatchGroup> step, entry, exit_;
  int64_t unknowns = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // Steady-state schedule: the groups of a pass one after another on one stream with programmatic
  // dependent launch (0), or as parallel graph branches joined before the next pass (1). Chosen at
  // creation by timing both graphs (trial_us: microseconds per step, serial / parallel).
  int concurrent = 0;
  double trial_us[2] = {0.0, 0.0};
  std::vector<cudaStream_t> side;   // capture streams of the parallel branches
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
};

namespace {

struct BatchTables {
  size_t off[2][5];
  double sc[2];
};

// PassArgs of problem i for one op, tile size P; returns the problem's tile count.
template <class T>
int batch_args(const etd_batch_s* b, const std::vector<BatchTables>& tabs, int i, int op, int axis, int f_in0,
               int f_in1, int f_out0, int f_out1, int P, const KernelInfo* k, PassArgs<T>& a) {
  memset(&a, 0, sizeof(a));
  a.user_slot = -1;
  a.ndim = 2;
  a.nx = b->nx[i];
  a.ny = b->ny[i];
  a.nz = 1;
  const T* base = static_cast<const T*>(b->tables);
  for (int d = 0; d < 3; ++d) {
    const int dd = d < 2 ? d : 0;
    a.zeta[d] = base + tabs[i].off[dd][2];
    a.ex[d] = base + tabs[i].off[dd][3];
    a.ec[d] = base + tabs[i].off[dd][4];
  }
  a.tw = base + tabs[i].off[axis][0];
  a.sn = base + tabs[i].off[axis][1];
  a.sc = (T)tabs[i].sc[axis];
  a.tau = (T)b->tau;
  a.c2 = (T)b->opt.c2;
  a.flin = (T)b->opt.flin;
  a.fcub = (T)b->opt.fcub;
  a.flog = (T)b->opt.flog;
  a.op = op;
  a.axis = axis;
  T* F = static_cast<T*>(b->ws) + b->field_off[i];
  const size_t fs = (size_t)b->nx[i] * b->ny[i];
  auto fld = [&](int f) -> T* { return f < 0 ? nullptr : F + (size_t)f * fs; };
  a.in0 = fld(f_in0);
  a.in1 = fld(f_in1);
  a.out0 = fld(f_out0);
  a.out1 = fld(f_out1);
  if (op == OP_ENTRY || op == OP_EXIT) a.user_slot = i;
  a.P = P;
  a.lp = pair_stride(*k, P);
  if (axis == 0) {
    a.npairs = b->ny[i] / 2;
    return (a.npairs + P - 1) / P;
  }
  a.tiles_x = b->nx[i] / (2 * P);
  return a.tiles_x;
}

template <class T>
etd_status batch_group_upload(etd_batch_s* b, const std::vector<BatchTables>& tabs, BatchGroup& g, int f_in0,
                              int f_in1, int f_out0, int f_out1, char*& aux_cursor) {
  const KernelInfo* k = find_pass_kernel((int)sizeof(T), g.N, g.axis == 0 ? b->oddx[g.inst[0]] : b->oddy[g.inst[0]]);
  std::vector<PassArgs<T>> descs(g.inst.size());
  std::vector<int2> map;
  for (size_t li = 0; li < g.inst.size(); ++li) {
    const int tiles = batch_args<T>(b, tabs, g.inst[li], g.op, g.axis, f_in0, f_in1, f_out0, f_out1, g.P, k, descs[li]);
    for (int t = 0; t < tiles; ++t) map.push_back(make_int2((int)li, t));
  }
  g.nctas = (int)map.size();
  g.smem = pass_smem_bytes(*k, g.P, g.nbuf);
  const size_t dbytes = descs.size() * sizeof(PassArgs<T>), mbytes = map.size() * sizeof(int2);
  g.d_descs = aux_cursor;
  aux_cursor += (dbytes + 255) & ~(size_t)255;
  g.d_map = aux_cursor;
  aux_cursor += (mbytes + 255) & ~(size_t)255;
  if (aux_cursor > static_cast<char*>(b->d_aux) + b->aux_bytes) return fail(ETD_ERR_CUDA, "batch descriptor area overflow");
  ETD_CUDA(cudaMemcpy(g.d_descs, descs.data(), dbytes, cudaMemcpyHostToDevice));
  ETD_CUDA(cudaMemcpy(g.d_map, map.data(), mbytes, cudaMemcpyHostToDevice));
  return ETD_OK;
}

etd_status batch_launch(const etd_batch_s* b, const BatchGroup& g, cudaStream_t s, bool pdl = true) {
  static const int use_pdl = env_int("ETD_PDL", 1);
  void* user = b->d_user;
  void* argv[3] = {const_cast<void**>(&g.d_descs), const_cast<void**>(&g.d_map), &user};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.nctas);
  cfg.blockDim = dim3((unsigned)(g.P * g.tpp));
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (use_pdl && pdl) ? 1 : 0;
  cudaError_t e = cudaLaunchKernelExC(&cfg, g.fn, argv);
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "batched kernel launch: %s", cudaGetErrorString(e));
  return ETD_OK;
}

struct BatchOp {
  int op, axis, in0, in1, out0, out1, kind, nbuf;
  double rw;
};

// Build every group of one op: instances grouped by the length of the transformed axis; the tile
// size is tuned once per (axis, length, buffers) and reused by later ops with the same shape.
template <class T>
etd_status batch_build_op(etd_batch_s* b, const std::vector<BatchTables>& tabs, const BatchOp& o,
                          std::vector<BatchGroup>& out, char*& aux, std::map<long long, int>& tuned, bool autotune) {
  std::map<int, std::vector<int>> by_len;
  for (int i = 0; i < b->count; ++i) by_len[o.axis == 0 ? b->nx[i] : b->ny[i]].push_back(i);
  for (auto& kv : by_len) {
    BatchGroup g;
    g.axis = o.axis;
    g.op = o.op;
    g.N = kv.first;
    g.inst = kv.second;
    g.nbuf = o.nbuf;
    g.kind = o.kind;
    const int odd = o.axis == 0 ? b->oddx[g.inst[0]] : b->oddy[g.inst[0]];
    const KernelInfo* k = find_pass_kernel((int)sizeof(T), g.N, odd);
    if (!k) return fail(ETD_ERR_UNSUPPORTED, "no kernel for axis length %d", g.N);
    g.fn = (o.op >= 0 && o.op < OP_COUNT && k->fn_batched_op[o.op]) ? k->fn_batched_op[o.op] : k->fn_batched;
    g.tpp = k->tpp;
    long long unk = 0;
    const int cut = b->periodic ? 0 : 1;
    for (int i : g.inst) unk += (long long)(b->nx[i] - cut) * (b->ny[i] - cut);
    g.alg_bytes = o.rw * (double)unk * sizeof(T);
    {
      cudaError_t e = cudaFuncSetAttribute(g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b->optin);
      if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    // candidate tile sizes: powers of two up to 512 threads, within the shared-memory budget, and
    // (strided passes) dividing every problem's x extent
    std::vector<int> cands;
    const size_t budget = (size_t)b->optin / (size_t)k->min_blocks - 2048;
    for (int P = 1; P * k->tpp <= 512; P *= 2) {
      if (pass_smem_bytes(*k, P, o.nbuf) > budget) break;
      bool ok = true;
      if (o.axis != 0)
        for (int i : g.inst) ok = ok && (b->nx[i] % (2 * P) == 0);
      if (ok) cands.push_back(P);
    }
    if (cands.empty()) return fail(ETD_ERR_UNSUPPORTED, "no tile size fits axis length %d", g.N);
    const long long key = ((long long)o.axis << 40) | ((long long)g.N << 8) | o.nbuf;
    auto it = tuned.find(key);
    if (it != tuned.end()) {
      g.P = it->second;
    } else if (!autotune || cands.size() == 1) {
      g.P = cands[cands.size() / 2];
      tuned[key] = g.P;
    } else {
      char* mark = aux;
      float best = 1e30f;
      int bestP = cands[0];
      cudaEvent_t e0, e1;
      ETD_CUDA(cudaEventCreate(&e0));
      ETD_CUDA(cudaEventCreate(&e1));
      for (int P : cands) {
        g.P = P;
        aux = mark;
        etd_status st = batch_group_upload<T>(b, tabs, g, o.in0, o.in1, o.out0, o.out1, aux);
        if (st != ETD_OK) return st;
        for (int w = 0; w < 2; ++w)
          if ((st = batch_launch(b, g, 0)) != ETD_OK) return st;
        ETD_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 5; ++r)
          if ((st = batch_launch(b, g, 0)) != ETD_OK) return st;
        ETD_CUDA(cudaEventRecord(e1, 0));
        ETD_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          bestP = P;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      aux = mark;
      g.P = bestP;
      tuned[key] = bestP;
    }
    etd_status st = batch_group_upload<T>(b, tabs, g, o.in0, o.in1, o.out0, o.out1, aux);
    if (st != ETD_OK) return st;
    out.push_back(g);
  }
  return ETD_OK;
}

// Captures G steady-state time steps into an executable graph. Serial schedule: every group on one
// stream, each launch with programmatic dependent launch on its predecessor. Parallel schedule: the
// groups of a pass (disjoint problems) as parallel branches forked from and joined into the capture
// stream, so a pass takes the time of its slowest group rather than the sum; no programmatic edges
// (the pass kernels' dependency wait then returns at once).
etd_status batch_capture(etd_batch_s* b, int G, bool parallel, cudaGraphExec_t* out) {
  *out = nullptr;
  if (!b->cap_stream) ETD_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  size_t widest = 1;
  for (size_t i = 0, j; i < b->step.size(); i = j) {
    for (j = i; j < b->step.size() && b->step[j].pass == b->step[i].pass; ++j) {}
    widest = std::max(widest, j - i);
  }
  if (parallel) {
    while (b->side.size() < widest) {
      cudaStream_t ss = nullptr;
      ETD_CUDA(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking));
      b->side.push_back(ss);
    }
    if (!b->ev_fork) ETD_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    while (b->ev_join.size() < widest) {
      cudaEvent_t ev = nullptr;
      ETD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      b->ev_join.push_back(ev);
    }
  }
  cudaGraph_t g = nullptr;
  ETD_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  etd_status st = ETD_OK;
  cudaError_t ce = cudaSuccess;
  for (int k = 0; k < G && st == ETD_OK && ce == cudaSuccess; ++k) {
    for (size_t i = 0, j; i < b->step.size() && st == ETD_OK && ce == cudaSuccess; i = j) {
      for (j = i; j < b->step.size() && b->step[j].pass == b->step[i].pass; ++j) {}
      if (!parallel || j - i == 1) {
        for (size_t q = i; q < j && st == ETD_OK; ++q) st = batch_launch(b, b->step[q], b->cap_stream, !parallel);
        continue;
      }
      if ((ce = cudaEventRecord(b->ev_fork, b->cap_stream)) != cudaSuccess) break;
      for (size_t q = i; q < j; ++q) {
        cudaStream_t ss = b->side[q - i];
        if ((ce = cudaStreamWaitEvent(ss, b->ev_fork, 0)) != cudaSuccess) break;
        if ((st = batch_launch(b, b->step[q], ss, false)) != ETD_OK) break;
        if ((ce = cudaEventRecord(b->ev_join[q - i], ss)) != cudaSuccess) break;
        if ((ce = cudaStreamWaitEvent(b->cap_stream, b->ev_join[q - i], 0)) != cudaSuccess) break;
      }
    }
  }
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  if (st != ETD_OK || ce != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != ETD_OK) return st;
    return fail(ETD_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(ce != cudaSuccess ? ce : e));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  return ETD_OK;
}

// Creation-time A/B of the two schedules (on the workspace, before any caller data): both graphs are
// built and timed, the faster one is kept for the runs.
etd_status batch_choose_schedule(etd_batch_s* b) {
  const int G = env_int("ETD_GRAPH_STEPS", 32);
  bool multi = false;
  for (size_t q = 1; q < b->step.size(); ++q) multi = multi || b->step[q].pass == b->step[q - 1].pass;
  if (G <= 0 || !multi) return ETD_OK;
  cudaGraphExec_t gx[2] = {nullptr, nullptr};
  etd_status st = ETD_OK;
  for (int m = 0; m < 2 && st == ETD_OK; ++m) st = batch_capture(b, G, m == 1, &gx[m]);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == ETD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = fail(ETD_ERR_CUDA, "event create");
  // alternate the schedules so that clock drift affects both alike; best of three per schedule
  float best[2] = {1e30f, 1e30f};
  for (int r = 0; r < 4 && st == ETD_OK; ++r)
    for (int m = 0; m < 2 && st == ETD_OK; ++m) {
      cudaError_t ce = cudaGraphLaunch(gx[m], b->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, b->cap_stream);
      if (ce == cudaSuccess) ce = cudaGraphLaunch(gx[m], b->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, b->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) {
        st = fail(ETD_ERR_CUDA, "schedule trial: %s", cudaGetErrorString(ce));
        break;
      }
      if (r > 0) best[m] = std::min(best[m], ms);
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st == ETD_OK) {
    const int pick = best[1] < best[0] ? 1 : 0;
    b->trial_us[0] = 1e3 * best[0] / G;
    b->trial_us[1] = 1e3 * best[1] / G;
    b->concurrent = pick;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = gx[pick];
    b->graph_steps = G;
    gx[pick] = nullptr;
  }
  for (cudaGraphExec_t x : gx)
    if (x) cudaGraphExecDestroy(x);
  return st;
}

template <class T>
etd_status batch_build(etd_batch_s* b) {
  // tables
  std::vector<T> h;
  std::vector<BatchTables> tabs(b->count);
  for (int i = 0; i < b->count; ++i) {
    const int n[2] = {b->nx[i], b->ny[i]};
    const double hh[2] = {b->hx[i], b->hy[i]};
    const int odd[2] = {b->oddx[i], b->oddy[i]};
    for (int a = 0; a < 2; ++a) {
      const KernelInfo* k = find_pass_kernel((int)sizeof(T), n[a], odd[a]);
      if (!k) return fail(ETD_ERR_UNSUPPORTED, "no kernel for axis length %d", n[a]);
      append_axis_tables<T>(k, n[a], hh[a], b->tau * b->Dv[i], b->opt.c2, h, tabs[i].off[a], b->periodic != 0);
      tabs[i].sc[a] = b->periodic ? 0.5 / sqrt((double)n[a]) : 0.5 * sqrt(2.0 / (double)n[a]);
    }
  }
  ETD_CUDA(cudaMalloc(&b->tables, h.size() * sizeof(T)));
  ETD_CUDA(cudaMemcpy(b->tables, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  // fields
  size_t total = 0;
  b->field_off.resize(b->count);
  for (int i = 0; i < b->count; ++i) {
    b->field_off[i] = total;
    total += 6 * (size_t)b->nx[i] * b->ny[i];   // V, N0, V2, P, N2, V~
    total = (total + 63) & ~(size_t)63;   // 256-byte aligned fields
    const int cut = b->periodic ? 0 : 1;
    b->unknowns += (int64_t)(b->nx[i] - cut) * (b->ny[i] - cut);
  }
  b->ws_bytes = total * sizeof(T);
  cudaError_t e = cudaMalloc(&b->ws, b->ws_bytes);
  if (e != cudaSuccess) return fail(ETD_ERR_OOM, "batch workspace of %zu bytes: %s", b->ws_bytes, cudaGetErrorString(e));
  ETD_CUDA(cudaMemset(b->ws, 0, b->ws_bytes));
  ETD_CUDA(cudaMalloc(&b->d_user, (size_t)b->count * sizeof(void*)));
  ETD_CUDA(cudaMemset(b->d_user, 0, (size_t)b->count * sizeof(void*)));
  // descriptor area: at most (ops) x (problems) descriptors and one map entry per tile at P = 1
  size_t tiles1 = 0;
  for (int i = 0; i < b->count; ++i) tiles1 += (size_t)b->ny[i] / 2 + (size_t)b->nx[i] / 2;
  const int nops = 8;
  b->aux_bytes = (size_t)nops * ((size_t)b->count * sizeof(PassArgs<T>) + tiles1 * sizeof(int2)) + (size_t)nops * 64 * 512;
  ETD_CUDA(cudaMalloc(&b->d_aux, b->aux_bytes));
  char* aux = static_cast<char*>(b->d_aux);
  // the step of a single plan with the spectral state V~ (y-transformed V): the stage passes read V~
  // instead of transforming V, the last pass writes both
  enum { V = 0, N0 = 1, V2 = 2, PF = 3, N2 = 4, VS = 5 };
  std::vector<BatchOp> ops;
  if (b->scheme == 2) {
    ops = {{OP_REACT, 0, V, -1, N0, -1, PK_REACT, 1, 2.0},
           {OP_S1S, 1, VS, N0, V2, PF, PK_S1, 2, 4.0},
           {OP_REACT, 0, V2, -1, N2, -1, PK_REACT, 1, 2.0},
           {OP_S2S, 1, N2, PF, V, VS, PK_S2, 2, 4.0}};
  } else {
    ops = {{OP_REACT, 0, V, -1, N0, -1, PK_REACT, 1, 2.0}, {OP_RK1S, 1, VS, N0, V, VS, PK_RK1, 2, 4.0}};
  }
  const bool autotune = env_int("ETD_AUTOTUNE", 1) != 0;
  std::map<long long, int> tuned;
  for (size_t oi = 0; oi < ops.size(); ++oi) {
    const size_t first = b->step.size();
    etd_status st = batch_build_op<T>(b, tabs, ops[oi], b->step, aux, tuned, autotune);
    if (st != ETD_OK) return st;
    for (size_t q = first; q < b->step.size(); ++q) b->step[q].pass = (int)oi;
  }
  const BatchOp ent{OP_ENTRY, 0, -1, -1, V, -1, PK_ENTRY_EXIT, 1, 2.0}, ext{OP_EXIT, 0, V, -1, -1, -1, PK_ENTRY_EXIT, 1, 2.0};
  const BatchOp ent_s{OP_TRANSFORM, 1, V, -1, VS, -1, PK_ENTRY_EXIT, 1, 2.0};
  etd_status st = batch_build_op<T>(b, tabs, ent, b->entry, aux, tuned, false);
  if (st != ETD_OK) return st;
  st = batch_build_op<T>(b, tabs, ent_s, b->entry, aux, tuned, false);
  if (st != ETD_OK) return st;
  st = batch_build_op<T>(b, tabs, ext, b->exit_, aux, tuned, false);
  if (st != ETD_OK) return st;
  if (b->opt.debug == ETD_DEBUG_BATCH_SERIAL || b->opt.debug == ETD_DEBUG_BATCH_PARALLEL) {
    b->concurrent = b->opt.debug == ETD_DEBUG_BATCH_PARALLEL;
  } else if (autotune) {
    etd_status st2 = batch_choose_schedule(b);
    if (st2 != ETD_OK) return st2;
  }
  // the autotuner ran passes on the workspace: restore the zero state the boundary slots rely on
  ETD_CUDA(cudaMemset(b->ws, 0, b->ws_bytes));
  ETD_CUDA(cudaDeviceSynchronize());
  return ETD_OK;
}

etd_status batch_run_steps(etd_batch_s* b, int64_t nsteps, cudaStream_t s) {
  const int G = env_int("ETD_GRAPH_STEPS", 32);
  int64_t done = 0;
  if (G > 0 && nsteps >= G) {
    if (!b->graph || b->graph_steps != G) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      b->graph_steps = 0;
      etd_status st = batch_capture(b, G, b->concurrent != 0, &b->graph);
      if (st != ETD_OK) return st;
      b->graph_steps = G;
    }
    for (; done + G <= nsteps; done += G) ETD_CUDA(cudaGraphLaunch(b->graph, s));
  }
  for (; done < nsteps; ++done)
    for (const BatchGroup& grp : b->step) {
      etd_status st = batch_launch(b, grp, s);
      if (st != ETD_OK) return st;
    }
  return ETD_OK;
}

}  // namespace

namespace {
// One mode per thread: the weights as the pass epilogues evaluate them, from inputs rounded to T.
template <class T>
__global__ void phi_weights_kernel(const double* __restrict__ zeta, const double* __restrict__ E,
                                   const double* __restrict__ Ec, double c2, long long n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned act = __activemask();
  const T z = (T)zeta[i];
  T p1, p2, rz;
  stage_phi12<T>(z, (T)E[i], act, p1, p2, rz);
  const T p1c = stage_phi1c<T>(z, (T)Ec[i], (T)c2, rz, act);
  out[3 * i] = (double)p1;
  out[3 * i + 1] = (double)p2;
  out[3 * i + 2] = (double)p1c;
}
}  // namespace

extern "C" {

etd_status etd_phi_weights(etd_dtype dtype, int64_t n, const double* zeta, const double* E, const double* Ec,
                           double c2, double* out) {
  g_last_error.clear();
  if (dtype != ETD_F32 && dtype != ETD_F64) return fail(ETD_ERR_INVALID_ARG, "dtype must be ETD_F32 or ETD_F64");
  if (n < 0) return fail(ETD_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (!zeta || !E || !Ec || !out)) return fail(ETD_ERR_INVALID_ARG, "NULL array");
  if (!(std::isfinite(c2) && c2 > 0 && c2 <= 1)) return fail(ETD_ERR_INVALID_ARG, "c2 must lie in (0, 1]");
  for (int64_t i = 0; i < n; ++i)
    if (!(std::isfinite(zeta[i]) && zeta[i] >= 0) || !std::isfinite(E[i]) || !std::isfinite(Ec[i]))
      return fail(ETD_ERR_INVALID_ARG, "zeta must be finite and >= 0, E and Ec finite (entry %lld)", (long long)i);
  if (n == 0) return ETD_OK;
  double* d = nullptr;
  const size_t in_bytes = 3 * (size_t)n * sizeof(double);
  cudaError_t e = cudaMalloc(&d, 2 * in_bytes);
  if (e != cudaSuccess) return fail(ETD_ERR_OOM, "device buffer: %s", cudaGetErrorString(e));
  etd_status st = ETD_OK;
  if ((e = cudaMemcpy(d, zeta, n * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d + n, E, n * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d + 2 * n, Ec, n * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
    st = fail(ETD_ERR_CUDA, "copy in: %s", cudaGetErrorString(e));
  } else {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (dtype == ETD_F32) phi_weights_kernel<float><<<blocks, 256>>>(d, d + n, d + 2 * n, c2, n, d + 3 * n);
    else phi_weights_kernel<double><<<blocks, 256>>>(d, d + n, d + 2 * n, c2, n, d + 3 * n);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaMemcpy(out, d + 3 * n, in_bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
      st = fail(ETD_ERR_CUDA, "phi weights: %s", cudaGetErrorString(e));
  }
  cudaFree(d);
  return st;
}

etd_status etd_options_default(etd_options* opt) {
  if (!opt) return fail(ETD_ERR_INVALID_ARG, "opt is NULL");
  opt->dtype = ETD_F64;
  opt->route = ETD_ROUTE_AUTO;
  opt->c2 = 0.5;
  opt->flin = 1.0;
  opt->fcub = -1.0;
  opt->debug = 0;
  opt->bc = ETD_BC_DIRICHLET;
  opt->flog = 0.0;
  return ETD_OK;
}

etd_status etd_plan_create(etd_plan* out, int ndim, const int64_t* N, const double* h, double D,
                           double tau, etd_scheme scheme, const etd_options* opt) {
  g_last_error.clear();
  if (!out) return fail(ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!N || !h) return fail(ETD_ERR_INVALID_ARG, "N or h is NULL");
  if (ndim != 2 && ndim != 3) return fail(ETD_ERR_INVALID_ARG, "ndim must be 2 or 3 (got %d)", ndim);
  if (scheme != ETD_ETDRK1 && scheme != ETD_ETDRK2) return fail(ETD_ERR_INVALID_ARG, "scheme must be 1 or 2");
  if (!(std::isfinite(D) && D > 0)) return fail(ETD_ERR_INVALID_ARG, "D must be finite and > 0");
  if (!(std::isfinite(tau) && tau > 0)) return fail(ETD_ERR_INVALID_ARG, "tau must be finite and > 0");
  etd_options o;
  etd_options_default(&o);
  if (opt) o = *opt;
  if (!(std::isfinite(o.c2) && o.c2 > 0 && o.c2 <= 1)) return fail(ETD_ERR_INVALID_ARG, "c2 must lie in (0, 1]");
  if (!std::isfinite(o.flin) || !std::isfinite(o.fcub) || !std::isfinite(o.flog))
    return fail(ETD_ERR_INVALID_ARG, "reaction coefficients must be finite");
  if (o.dtype != ETD_F32 && o.dtype != ETD_F64) return fail(ETD_ERR_INVALID_ARG, "dtype must be ETD_F32 or ETD_F64");
  if (o.route != ETD_ROUTE_AUTO && o.route != ETD_ROUTE_FFT && o.route != ETD_ROUTE_FFT_HALF &&
      o.route != ETD_ROUTE_GEMM_TF32 && o.route != ETD_ROUTE_GEMM_BF16X3 && o.route != ETD_ROUTE_FFT_SPLIT)
    return fail(ETD_ERR_INVALID_ARG, "unknown route");
  if (o.bc != ETD_BC_DIRICHLET && o.bc != ETD_BC_PERIODIC) return fail(ETD_ERR_INVALID_ARG, "unknown boundary condition");
  const bool gemm = o.route == ETD_ROUTE_GEMM_TF32 || o.route == ETD_ROUTE_GEMM_BF16X3;
  if (gemm && o.dtype != ETD_F32) return fail(ETD_ERR_INVALID_ARG, "the GEMM routes compute in FP32 (dtype ETD_F32)");
  for (int a = 0; a < ndim; ++a) {
    if (N[a] < 2) return fail(ETD_ERR_INVALID_ARG, "N[%d] = %lld < 2", a, (long long)N[a]);
    if (N[a] % 2) return fail(ETD_ERR_INVALID_ARG, "N[%d] = %lld must be even", a, (long long)N[a]);
    if (!(std::isfinite(h[a]) && h[a] > 0)) return fail(ETD_ERR_INVALID_ARG, "h[%d] must be finite and > 0", a);
  }
  for (int a = 0; a < ndim; ++a)
    if (!supported_length(N[a]))
      return fail(ETD_ERR_UNSUPPORTED, "N[%d] = %lld: supported lengths are 2^k (4..2048) and 3*2^k (6..1536)", a,
                  (long long)N[a]);
  if (gemm)
    for (int a = 0; a < ndim; ++a)
      if (N[a] % 32)
        return fail(ETD_ERR_UNSUPPORTED, "N[%d] = %lld: the GEMM routes need multiples of 32", a, (long long)N[a]);
  if (o.flog != 0.0 && !gemm && o.bc != ETD_BC_PERIODIC)
    return fail(ETD_ERR_UNSUPPORTED, "the artanh reaction term runs on periodic plans and on the GEMM routes");
  etd_plan_s* pl = new etd_plan_s();
  pl->periodic = o.bc == ETD_BC_PERIODIC;
  pl->ndim = ndim;
  for (int a = 0; a < ndim; ++a) {
    pl->N[a] = N[a];
    pl->h[a] = h[a];
  }
  pl->D = D;
  pl->tau = tau;
  pl->scheme = scheme;
  pl->opt = o;
  pl->elem = (o.dtype == ETD_F32) ? 4 : 8;
  for (int a = 0; a < ndim; ++a) {
    // FP32: the odd extension keeps rounding at log N; AUTO uses it from N = 512 up and the
    // half-length recurrence (sqrt(N/2) eps <= 11 eps) below, where it is twice as fast.
    // Periodic axes: the Hartley variant (a plain length-N FFT, rounding like log N) on every route.
    if (pl->periodic) pl->odd[a] = V_HART;
    else if (o.dtype != ETD_F32 || o.route == ETD_ROUTE_FFT_HALF) pl->odd[a] = V_REC;
    else if (o.route == ETD_ROUTE_FFT) pl->odd[a] = V_ODD;
    else pl->odd[a] = N[a] >= 512 ? V_ODD : V_REC;
  }
  // ETD_ROUTE_FFT_SPLIT: FP32 Dirichlet axes of length 1024 take the split-radix kernels (the strided
  // passes need an x extent that is a multiple of 4); every other axis the AUTO choice.
  for (int a = 0; a < ndim; ++a)
    pl->split[a] = (o.dtype == ETD_F32 && !pl->periodic && o.route == ETD_ROUTE_FFT_SPLIT && N[a] == SPLIT_N &&
                    (a == 0 || N[0] % 4 == 0)) ? 1 : 0;
  pl->nx = (int)N[0];
  pl->ny = (int)N[1];
  pl->nz = ndim == 3 ? (int)N[2] : 1;
  pl->nfield = (size_t)pl->nx * pl->ny * pl->nz;
  const int64_t cut = pl->periodic ? 0 : 1;
  pl->unknowns = (N[0] - cut) * (N[1] - cut) * (ndim == 3 ? N[2] - cut : 1);
  auto bail = [&](etd_status s) {
    etd_destroy(pl);
    return s;
  };
  if (cudaGetDevice(&pl->device) != cudaSuccess) return bail(fail(ETD_ERR_CUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
  const size_t fbytes = pl->nfield * pl->elem;
  // FFT routes keep V~ (a sixth field), except where the last axis runs the split-radix kernels,
  // which have no stage passes on it
  pl->spec = !gemm && !pl->split[ndim - 1];
  const int nf = pl->spec ? 6 : 5;
  pl->ws_bytes = nf * fbytes;
  cudaError_t e = cudaMalloc(&pl->ws, pl->ws_bytes);
  if (e != cudaSuccess) return bail(fail(ETD_ERR_OOM, "workspace of %zu bytes: %s", pl->ws_bytes, cudaGetErrorString(e)));
  e = cudaMemset(pl->ws, 0, pl->ws_bytes);
  if (e != cudaSuccess) return bail(fail(ETD_ERR_CUDA, "memset: %s", cudaGetErrorString(e)));
  for (int f = 0; f < nf; ++f) pl->F[f] = static_cast<char*>(pl->ws) + f * fbytes;
  etd_status st = (pl->elem == 4) ? upload_tables<float>(pl) : upload_tables<double>(pl);
  if (st != ETD_OK) return bail(st);
  // per-mode phi-function weights of the y passes of 2D plans on the FFT routes (at most 64 MiB): FP32
  // plans, and FP64 plans whose y axis runs the FP64 operation-fixed kernels (N = 1024), which read them
  const size_t coef_bytes = pl->nfield * (pl->scheme == 2 ? 3 : 1) * (size_t)pl->elem;
  if (ndim == 2 && !pl->periodic && !gemm && coef_bytes <= ((size_t)64 << 20)) {
    if (pl->elem == 4) st = upload_coef_tables<float>(pl);
    else if (pl->odd[1] == V_REC && N[1] == 1024) st = upload_coef_tables<double>(pl);
    if (st != ETD_OK) return bail(st);
  }
  if (gemm) {
    pl->gemm = 1 + (o.route == ETD_ROUTE_GEMM_TF32 ? GR_TF32 : GR_BF16X3);
    if ((st = upload_gemm_tables(pl)) != ETD_OK) return bail(st);
    st = build_step_gemm(pl);
  } else {
    st = (pl->elem == 4) ? build_step<float>(pl) : build_step<double>(pl);
  }
  if (st != ETD_OK) return bail(st);
  pl->mon_blocks = 2 * pl->num_sms;
  e = cudaMalloc(&pl->mon_part, (size_t)pl->mon_blocks * 4 * sizeof(double) + (size_t)pl->mon_blocks * sizeof(long long) +
                                    8 * sizeof(double));
  if (e != cudaSuccess) return bail(fail(ETD_ERR_OOM, "monitor scratch: %s", cudaGetErrorString(e)));
  pl->mon_bad = reinterpret_cast<long long*>(pl->mon_part + 4 * pl->mon_blocks);
  pl->mon_out = reinterpret_cast<double*>(pl->mon_bad + pl->mon_blocks);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return bail(fail(ETD_ERR_CUDA, "plan setup: %s", cudaGetErrorString(e)));
  *out = pl;
  return ETD_OK;
}

etd_status etd_run_from(etd_plan pl, void* u, int64_t nsteps, double t0, void* stream) {
  if (!pl || !u) return fail(ETD_ERR_INVALID_ARG, "plan or u is NULL");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  if (!std::isfinite(t0)) return fail(ETD_ERR_INVALID_ARG, "t0 must be finite");
  if (nsteps == 0) return ETD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pl->src_on) {
    source_clock_kernel<<<1, 1, 0, s>>>(static_cast<unsigned long long*>(pl->clock),
                                         reinterpret_cast<double*>(static_cast<char*>(pl->clock) + 8), t0);
    ETD_CUDA(cudaGetLastError());
  }
  std::vector<Launch> ent, ext;
  etd_status st = entry_exit_any(pl, true, u, ent);
  if (st != ETD_OK) return st;
  st = entry_exit_any(pl, false, u, ext);
  if (st != ETD_OK) return st;
  for (const Launch& L : ent)
    if ((st = launch(L, s)) != ETD_OK) return st;
  st = pl->bnd_on ? run_steps_boundary(pl, nsteps, t0, s) : run_steps(pl, nsteps, s);
  if (st != ETD_OK) return st;
  for (const Launch& L : ext)
    if ((st = launch(L, s)) != ETD_OK) return st;
  return ETD_OK;
}

etd_status etd_run(etd_plan pl, void* u, int64_t nsteps, void* stream) {
  return etd_run_from(pl, u, nsteps, 0.0, stream);
}

etd_status etd_step(etd_plan pl, void* u, void* stream) { return etd_run(pl, u, 1, stream); }

etd_status etd_set_source(etd_plan pl, double amp, double rate, const double* gx, const double* gy,
                          const double* gz) {
  if (!pl) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
  if (!gx && !gy && !gz) {   // remove the source
    if (!pl->src_on) return ETD_OK;
    pl->src_on = false;
  } else {
    const double* g[3] = {gx, gy, gz};
    for (int d = 0; d < pl->ndim; ++d)
      if (!g[d]) return fail(ETD_ERR_INVALID_ARG, "one profile per axis is needed (axis %d is NULL)", d);
    if (pl->ndim == 2 && gz) return fail(ETD_ERR_INVALID_ARG, "gz must be NULL for a 2D plan");
    if (!std::isfinite(amp) || !std::isfinite(rate)) return fail(ETD_ERR_INVALID_ARG, "amp and rate must be finite");
    if (pl->gemm) return fail(ETD_ERR_UNSUPPORTED, "sources are supported on the FFT routes");
    const int n[3] = {pl->nx, pl->ny, pl->nz};
    const int cut = pl->periodic ? 0 : 1;   // profile entries per axis: n - cut
    for (int d = 0; d < pl->ndim; ++d)
      for (int i = 0; i < n[d] - cut; ++i)
        if (!std::isfinite(g[d][i])) return fail(ETD_ERR_INVALID_ARG, "profile %d entry %d is not finite", d, i);
    // x: the spectral profile S_x g_x (orthonormal DST-I) or H_x g_x (orthonormal DHT), FP64, the
    // product's index reduced mod 2N (mod N); y, z: the nodal profiles; Dirichlet index 0 = 0
    const size_t tot = (size_t)pl->nx + pl->ny + pl->nz;
    std::vector<double> h(tot, 0.0);
    {
      const long long N = n[0];
      if (pl->periodic) {
        const double s0 = 1.0 / std::sqrt((double)N);
        for (long long k = 0; k < N; ++k) {
          double acc = 0.0;
          for (long long j = 0; j < N; ++j) {
            const double t = 2.0 * M_PI * (double)((j * k) % N) / (double)N;
            acc += g[0][j] * (std::cos(t) + std::sin(t));
          }
          h[k] = s0 * acc;
        }
      } else {
        const double s0 = std::sqrt(2.0 / (double)N);
        for (long long k = 1; k < N; ++k) {
          double acc = 0.0;
          for (long long j = 1; j < N; ++j) acc += g[0][j - 1] * std::sin(M_PI * (double)((j * k) % (2 * N)) / (double)N);
          h[k] = s0 * acc;
        }
      }
    }
    size_t off = (size_t)n[0];
    for (int d = 1; d < pl->ndim; ++d) {
      for (int i = cut; i < n[d]; ++i) h[off + i] = g[d][i - cut];
      off += n[d];
    }
    if (!pl->src_tab) ETD_CUDA(cudaMalloc(&pl->src_tab, tot * pl->elem));
    if (!pl->clock) ETD_CUDA(cudaMalloc(&pl->clock, 16));
    if (pl->elem == 4) {
      std::vector<float> f(h.begin(), h.end());
      ETD_CUDA(cudaMemcpy(pl->src_tab, f.data(), tot * 4, cudaMemcpyHostToDevice));
    } else {
      ETD_CUDA(cudaMemcpy(pl->src_tab, h.data(), tot * 8, cudaMemcpyHostToDevice));
    }
    ETD_CUDA(cudaMemset(pl->clock, 0, 16));
    pl->src_on = true;
    pl->src_amp = amp;
    pl->src_rate = rate;
  }
  destroy_graph(pl);
  etd_status st = pl->elem == 4 ? build_step<float>(pl) : build_step<double>(pl);
  if (st != ETD_OK) return st;
  if (pl->elem == 4) apply_source<float>(pl);
  else apply_source<double>(pl);
  return ETD_OK;
}

etd_status etd_boundary_count(etd_plan pl, int64_t* count) {
  if (!pl || !count) return fail(ETD_ERR_INVALID_ARG, "plan or count is NULL");
  if (pl->periodic) return fail(ETD_ERR_INVALID_ARG, "a periodic plan has no boundary");
  const int64_t Nx = pl->N[0], Ny = pl->N[1], Nz = pl->ndim == 3 ? pl->N[2] : 0;
  *count = pl->ndim == 3 ? 2 * (Nz + 1) * (Ny + 1) + 2 * (Nz + 1) * (Nx + 1) + 2 * (Ny + 1) * (Nx + 1)
                         : 2 * (Ny + 1) + 2 * (Nx + 1);
  return ETD_OK;
}

etd_status etd_set_boundary(etd_plan pl, etd_boundary_fn fn, void* ctx) {
  if (!pl) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
  if (pl->periodic) return fail(ETD_ERR_INVALID_ARG, "a periodic plan has no boundary");
  if (pl->gemm) return fail(ETD_ERR_UNSUPPORTED, "boundary data are supported on the FFT routes");
  if (!fn) {
    if (!pl->bnd_on) return ETD_OK;
    pl->bnd_on = false;
  } else {
    int64_t count = 0;
    etd_status st = etd_boundary_count(pl, &count);
    if (st != ETD_OK) return st;
    if (!pl->bnd_host) {
      const size_t bytes = 4 * (size_t)count * sizeof(double);   // two stages x (values, derivatives)
      ETD_CUDA(cudaMallocHost(&pl->bnd_host, bytes));
      ETD_CUDA(cudaMalloc(&pl->bnd_dev, bytes));
      ETD_CUDA(cudaMalloc(&pl->bnd_field, pl->nfield * pl->elem));
      // 1 / lambda^A per mode, lambda^A_i = (h/3)(2 + cos(i pi / N)) (mode 0: unused, 0)
      std::vector<double> ia((size_t)pl->nx + pl->ny + pl->nz, 0.0);
      size_t off = 0;
      const int n[3] = {pl->nx, pl->ny, pl->nz};
      for (int d = 0; d < pl->ndim; ++d) {
        for (int i = 1; i < n[d]; ++i)
          ia[off + i] = 3.0 / (pl->h[d] * (2.0 + cos(M_PI * (double)i / (double)n[d])));
        off += n[d];
      }
      ETD_CUDA(cudaMalloc(&pl->bnd_ia, ia.size() * sizeof(double)));
      ETD_CUDA(cudaMemcpy(pl->bnd_ia, ia.data(), ia.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    pl->bnd_count = count;
    pl->bnd_fn = fn;
    pl->bnd_ctx = ctx;
    pl->bnd_on = true;
  }
  destroy_graph(pl);
  etd_status st = pl->elem == 4 ? build_step<float>(pl) : build_step<double>(pl);
  if (st != ETD_OK) return st;
  if (pl->elem == 4) apply_source<float>(pl);
  else apply_source<double>(pl);
  return ETD_OK;
}

etd_status etd_run_host(etd_plan pl, void* u_host, int64_t nsteps, void* stream) {
  if (!pl || !u_host) return fail(ETD_ERR_INVALID_ARG, "plan or u_host is NULL");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)pl->unknowns * pl->elem;
  if (!pl->host_dev) ETD_CUDA(cudaMalloc(&pl->host_dev, bytes));
  ETD_CUDA(cudaMemcpyAsync(pl->host_dev, u_host, bytes, cudaMemcpyHostToDevice, s));
  etd_status st = etd_run(pl, pl->host_dev, nsteps, stream);
  if (st != ETD_OK) return st;
  ETD_CUDA(cudaMemcpyAsync(u_host, pl->host_dev, bytes, cudaMemcpyDeviceToHost, s));
  ETD_CUDA(cudaStreamSynchronize(s));
  return check_dev_err(pl);
}

etd_status etd_apply_dst(etd_plan pl, int axis, const void* in, void* out, void* stream) {
  if (!pl || !in || !out) return fail(ETD_ERR_INVALID_ARG, "plan, in or out is NULL");
  if (axis < 0 || axis >= pl->ndim) return fail(ETD_ERR_INVALID_ARG, "axis %d out of range", axis);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Launch L;
  etd_status st;
  void* F0 = pl->F[0];
  auto mk = [&](int op, int ax, const void* i0, void* o0) -> etd_status {
    return pl->elem == 4 ? make_launch<float>(pl, op, ax, i0, nullptr, o0, nullptr, PK_PACK, 2, L)
                         : make_launch<double>(pl, op, ax, i0, nullptr, o0, nullptr, PK_PACK, 2, L);
  };
  if ((st = mk(OP_PACK, 0, in, F0)) != ETD_OK) return st;
  if ((st = launch(L, s)) != ETD_OK) return st;
  if ((st = mk(OP_TRANSFORM, axis, F0, F0)) != ETD_OK) return st;
  if ((st = launch(L, s)) != ETD_OK) return st;
  if ((st = mk(OP_UNPACK, 0, F0, out)) != ETD_OK) return st;
  if ((st = launch(L, s)) != ETD_OK) return st;
  return ETD_OK;
}

etd_status etd_monitor(etd_plan pl, const void* u, etd_monitors* out, void* stream) {
  if (!pl || !u || !out) return fail(ETD_ERR_INVALID_ARG, "plan, u or out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MonitorGeom g;
  g.ndim = pl->ndim;
  for (int a = 0; a < 3; ++a) {
    g.m[a] = a < pl->ndim ? (int)pl->N[a] - (pl->periodic ? 0 : 1) : 1;
    g.h[a] = a < pl->ndim ? pl->h[a] : 1.0;
  }
  g.D = pl->D;
  g.periodic = pl->periodic;
  g.flin = pl->opt.flin;
  g.fcub = pl->opt.fcub;
  g.flog = pl->opt.flog;
  if (pl->elem == 4)
    monitor_partial_kernel<float><<<pl->mon_blocks, 256, 0, s>>>(static_cast<const float*>(u), g, pl->mon_part, pl->mon_bad);
  else
    monitor_partial_kernel<double><<<pl->mon_blocks, 256, 0, s>>>(static_cast<const double*>(u), g, pl->mon_part, pl->mon_bad);
  ETD_CUDA(cudaGetLastError());
  monitor_final_kernel<<<1, 256, 0, s>>>(pl->mon_part, pl->mon_bad, pl->mon_blocks, pl->mon_out,
                                         reinterpret_cast<long long*>(pl->mon_out + 3));
  ETD_CUDA(cudaGetLastError());
  double hbuf[4];
  ETD_CUDA(cudaMemcpyAsync(hbuf, pl->mon_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ETD_CUDA(cudaStreamSynchronize(s));
  out->mass = hbuf[0];
  out->energy = hbuf[1];
  out->maxabs = hbuf[2];
  long long bad;
  memcpy(&bad, &hbuf[3], sizeof(bad));
  out->nonfinite = bad;
  etd_status st = check_dev_err(pl);
  if (st != ETD_OK) return st;
  if (bad) return fail(ETD_ERR_NONFINITE, "%lld non-finite values", bad);
  return ETD_OK;
}

etd_status etd_run_profiled(etd_plan pl, void* u, int64_t nsteps, void* stream, double* ms, int64_t* cnt) {
  if (!pl || !u || !ms || !cnt) return fail(ETD_ERR_INVALID_ARG, "NULL argument");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  if (pl->bnd_on) return fail(ETD_ERR_UNSUPPORTED, "profiled runs take homogeneous boundary data");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < ETD_NUM_PASS_KINDS; ++k) {
    ms[k] = 0;
    cnt[k] = 0;
  }
  if (pl->src_on) {
    source_clock_kernel<<<1, 1, 0, s>>>(static_cast<unsigned long long*>(pl->clock),
                                         reinterpret_cast<double*>(static_cast<char*>(pl->clock) + 8), 0.0);
    ETD_CUDA(cudaGetLastError());
  }
  std::vector<Launch> all, ent, ext;
  etd_status st = entry_exit_any(pl, true, u, ent);
  if (st != ETD_OK) return st;
  st = entry_exit_any(pl, false, u, ext);
  if (st != ETD_OK) return st;
  all = ent;
  for (int64_t i = 0; i < nsteps; ++i) all.insert(all.end(), pl->step.begin(), pl->step.end());
  all.insert(all.end(), ext.begin(), ext.end());
  std::vector<cudaEvent_t> ev(all.size() + 1);
  for (auto& e : ev) ETD_CUDA(cudaEventCreate(&e));
  ETD_CUDA(cudaEventRecord(ev[0], s));
  for (size_t i = 0; i < all.size(); ++i) {
    if ((st = launch(all[i], s)) != ETD_OK) break;
    ETD_CUDA(cudaEventRecord(ev[i + 1], s));
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == ETD_OK && e == cudaSuccess) {
    for (size_t i = 0; i < all.size(); ++i) {
      float t = 0;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[all[i].kind] += t;
      cnt[all[i].kind] += 1;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (st != ETD_OK) return st;
  if (e != cudaSuccess) return fail(ETD_ERR_CUDA, "profiled run: %s", cudaGetErrorString(e));
  return ETD_OK;
}

etd_status etd_get_plan_info(etd_plan pl, etd_plan_info* info) {
  if (!pl || !info) return fail(ETD_ERR_INVALID_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->ndim = pl->ndim;
  for (int a = 0; a < 3; ++a) info->N[a] = a < pl->ndim ? pl->N[a] : 1;
  info->unknowns = pl->unknowns;
  info->workspace_bytes = (int64_t)pl->ws_bytes;
  info->kernels_per_step = (int)pl->step.size();
  double b = 0;
  for (const Launch& L : pl->step) b += L.alg_bytes;
  info->bytes_per_step = b;
  info->dtype = pl->opt.dtype;
  info->scheme = pl->scheme;
  return ETD_OK;
}

const char* etd_pass_kind_name(int k) {
  return (k >= 0 && k < ETD_NUM_PASS_KINDS) ? kPassKindNames[k] : nullptr;
}

etd_status etd_destroy(etd_plan pl) {
  if (!pl) return ETD_OK;
  destroy_graph(pl);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (pl->ws) cudaFree(pl->ws);
  if (pl->tables) cudaFree(pl->tables);
  if (pl->coef) cudaFree(pl->coef);
  if (pl->host_dev) cudaFree(pl->host_dev);
  if (pl->mon_part) cudaFree(pl->mon_part);
  if (pl->gtab) cudaFree(pl->gtab);
  if (pl->src_tab) cudaFree(pl->src_tab);
  if (pl->clock) cudaFree(pl->clock);
  if (pl->dev_err) cudaFree(pl->dev_err);
  if (pl->bnd_host) cudaFreeHost(pl->bnd_host);
  if (pl->bnd_dev) cudaFree(pl->bnd_dev);
  if (pl->bnd_field) cudaFree(pl->bnd_field);
  if (pl->bnd_ia) cudaFree(pl->bnd_ia);
  delete pl;
  return ETD_OK;
}

etd_status etd_batch_create(etd_batch* out, int count, const int64_t* N, const double* h, const double* D, double tau,
                            etd_scheme scheme, const etd_options* opt) {
  g_last_error.clear();
  if (!out) return fail(ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count <= 0) return fail(ETD_ERR_INVALID_ARG, "count must be positive");
  if (!N || !h || !D) return fail(ETD_ERR_INVALID_ARG, "N, h or D is NULL");
  if (scheme != ETD_ETDRK1 && scheme != ETD_ETDRK2) return fail(ETD_ERR_INVALID_ARG, "scheme must be 1 or 2");
  if (!(std::isfinite(tau) && tau > 0)) return fail(ETD_ERR_INVALID_ARG, "tau must be finite and > 0");
  etd_options o;
  etd_options_default(&o);
  if (opt) o = *opt;
  if (!(std::isfinite(o.c2) && o.c2 > 0 && o.c2 <= 1)) return fail(ETD_ERR_INVALID_ARG, "c2 must lie in (0, 1]");
  if (!std::isfinite(o.flin) || !std::isfinite(o.fcub)) return fail(ETD_ERR_INVALID_ARG, "reaction coefficients must be finite");
  if (o.dtype != ETD_F32 && o.dtype != ETD_F64) return fail(ETD_ERR_INVALID_ARG, "dtype must be ETD_F32 or ETD_F64");
  if (o.route != ETD_ROUTE_AUTO && o.route != ETD_ROUTE_FFT && o.route != ETD_ROUTE_FFT_HALF &&
      o.route != ETD_ROUTE_GEMM_TF32 && o.route != ETD_ROUTE_GEMM_BF16X3 && o.route != ETD_ROUTE_FFT_SPLIT)
    return fail(ETD_ERR_INVALID_ARG, "unknown route");
  const bool gemm = o.route == ETD_ROUTE_GEMM_TF32 || o.route == ETD_ROUTE_GEMM_BF16X3;
  if (gemm) return fail(ETD_ERR_UNSUPPORTED, "batches run the FFT routes only");
  if (o.bc != ETD_BC_DIRICHLET && o.bc != ETD_BC_PERIODIC) return fail(ETD_ERR_INVALID_ARG, "unknown boundary condition");
  if (!std::isfinite(o.flog)) return fail(ETD_ERR_INVALID_ARG, "reaction coefficients must be finite");
  if (o.flog != 0.0 && o.bc != ETD_BC_PERIODIC)
    return fail(ETD_ERR_UNSUPPORTED, "the artanh reaction term runs on periodic batches only");
  for (int i = 0; i < count; ++i) {
    for (int a = 0; a < 2; ++a) {
      const int64_t n = N[2 * i + a];
      if (n < 2 || n % 2) return fail(ETD_ERR_INVALID_ARG, "problem %d: N[%d] = %lld must be even and >= 2", i, a, (long long)n);
      if (!(std::isfinite(h[2 * i + a]) && h[2 * i + a] > 0)) return fail(ETD_ERR_INVALID_ARG, "problem %d: h[%d] must be > 0", i, a);
      if (!supported_length(n)) return fail(ETD_ERR_UNSUPPORTED, "problem %d: N[%d] = %lld has no kernel", i, a, (long long)n);
    }
    if (!(std::isfinite(D[i]) && D[i] > 0)) return fail(ETD_ERR_INVALID_ARG, "problem %d: D must be finite and > 0", i);
  }
  etd_batch_s* b = new etd_batch_s();
  b->count = count;
  b->scheme = scheme;
  b->opt = o;
  b->periodic = o.bc == ETD_BC_PERIODIC;
  b->tau = tau;
  b->elem = o.dtype == ETD_F32 ? 4 : 8;
  for (int i = 0; i < count; ++i) {
    b->nx.push_back((int)N[2 * i]);
    b->ny.push_back((int)N[2 * i + 1]);
    b->hx.push_back(h[2 * i]);
    b->hy.push_back(h[2 * i + 1]);
    b->Dv.push_back(D[i]);
    auto odd_of = [&](int64_t n) {
      if (o.bc == ETD_BC_PERIODIC) return (int)V_HART;
      return (o.dtype != ETD_F32 || o.route == ETD_ROUTE_FFT_HALF) ? 0 : (o.route == ETD_ROUTE_FFT ? 1 : (n >= 512 ? 1 : 0));
    };
    b->oddx.push_back(odd_of(N[2 * i]));
    b->oddy.push_back(odd_of(N[2 * i + 1]));
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return fail(ETD_ERR_CUDA, "no CUDA device");
  }
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaDeviceGetAttribute(&b->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  etd_status st = b->elem == 4 ? batch_build<float>(b) : batch_build<double>(b);
  if (st != ETD_OK) {
    etd_batch_destroy(b);
    return st;
  }
  *out = b;
  return ETD_OK;
}

etd_status etd_batch_run(etd_batch b, void* const* u, int64_t nsteps, void* stream) {
  if (!b || !u) return fail(ETD_ERR_INVALID_ARG, "batch or u is NULL");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  for (int i = 0; i < b->count; ++i)
    if (!u[i]) return fail(ETD_ERR_INVALID_ARG, "u[%d] is NULL", i);
  if (nsteps == 0) return ETD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // pageable source: the copy is staged before the call returns, so u may be reused at once
  ETD_CUDA(cudaMemcpyAsync(b->d_user, u, (size_t)b->count * sizeof(void*), cudaMemcpyHostToDevice, s));
  etd_status st;
  for (const BatchGroup& g : b->entry)
    if ((st = batch_launch(b, g, s)) != ETD_OK) return st;
  if ((st = batch_run_steps(b, nsteps, s)) != ETD_OK) return st;
  for (const BatchGroup& g : b->exit_)
    if ((st = batch_launch(b, g, s)) != ETD_OK) return st;
  return ETD_OK;
}

etd_status etd_batch_info(etd_batch b, int64_t* unknowns, int* launches_per_step, int* tile_pairs, int max_groups) {
  if (!b) return fail(ETD_ERR_INVALID_ARG, "batch is NULL");
  if (unknowns) *unknowns = b->unknowns;
  if (launches_per_step) *launches_per_step = (int)b->step.size();
  if (tile_pairs)
    for (int i = 0; i < max_groups && i < (int)b->step.size(); ++i) tile_pairs[i] = b->step[i].P;
  return ETD_OK;
}

etd_status etd_batch_schedule(etd_batch b, int* parallel, double* us_serial, double* us_parallel) {
  if (!b) return fail(ETD_ERR_INVALID_ARG, "batch is NULL");
  if (parallel) *parallel = b->concurrent;
  if (us_serial) *us_serial = b->trial_us[0];
  if (us_parallel) *us_parallel = b->trial_us[1];
  return ETD_OK;
}

etd_status etd_batch_destroy(etd_batch b) {
  if (!b) return ETD_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaStream_t ss : b->side) cudaStreamDestroy(ss);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (cudaEvent_t ev : b->ev_join) cudaEventDestroy(ev);
  if (b->ws) cudaFree(b->ws);
  if (b->tables) cudaFree(b->tables);
  if (b->d_user) cudaFree(b->d_user);
  if (b->d_aux) cudaFree(b->d_aux);
  delete b;
  return ETD_OK;
}

const char* etd_status_string(etd_status s) {
  switch (s) {
    case ETD_OK: return "ok";
    case ETD_ERR_INVALID_ARG: return "invalid argument";
    case ETD_ERR_UNSUPPORTED: return "unsupported";
    case ETD_ERR_CUDA: return "CUDA error";
    case ETD_ERR_OOM: return "out of memory";
    case ETD_ERR_NONFINITE: return "non-finite values";
    case ETD_ERR_TIMEOUT: return "a device wait ran out";
  }
  return "unknown status";
}

const char* etd_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
