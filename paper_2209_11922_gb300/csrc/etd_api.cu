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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/etd.h"
#include "monitor.cuh"
#include "pass_kernel.cuh"

namespace etd {
// registry of instantiated pass kernels (generated per (type, N) translation units)
const KernelInfo* find_pass_kernel(int elem, int N, int odd);
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
                PK_PACK = 6, PK_MONITOR = 7 };
const char* kPassKindNames[ETD_NUM_PASS_KINDS] = {"entry_exit", "x_react", "transform", "stage1_etdrk2",
                                                   "stage2_etdrk2", "stage_etdrk1", "pack", "monitor"};

struct Launch {
  const void* fn;
  dim3 grid, block;
  size_t smem;
  int kind;
  alignas(16) unsigned char args[sizeof(PassArgs<double>)];
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
  int odd[3] = {0, 0, 0};  // DST variant per axis: 1 odd extension, 0 half-length recurrence
  int nx = 1, ny = 1, nz = 1;
  size_t nfield = 0;       // pitched elements per field
  int64_t unknowns = 0;    // interior unknowns
  int device = 0;
  int num_sms = 148;
  void* ws = nullptr;      // fields
  void* F[5] = {};         // V, N0, V2, P, N2
  void* tables = nullptr;
  const void* tw[3] = {};
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
};

namespace {

template <class T>
void fill_common(const etd_plan_s* pl, PassArgs<T>& a) {
  memset(&a, 0, sizeof(a));
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
}

// Build one pass launch. fields are indices into F (or -1 for a user pointer given later).
template <class T>
etd_status make_launch(etd_plan_s* pl, int op, int axis, const void* in0, const void* in1, void* out0,
                       void* out1, int kind, double fields_rw, Launch& L) {
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
  const bool two = (op == OP_RK1 || op == OP_S1 || op == OP_S2);
  const int maxp = 512 / k->tpp > 0 ? 512 / k->tpp : 1;
  int P = 1;
  long long grid = 0;
  if (axis == 0) {
    a.npairs = pl->ny * pl->nz / 2;
    P = env_int("ETD_PAIRS_X", 0);
    if (P <= 0) {
      P = maxp;
      while (P > 1 && (a.npairs + P - 1) / P < 2 * pl->num_sms) P /= 2;
    }
    if (P > maxp) P = maxp;
    grid = (a.npairs + P - 1) / P;
  } else {
    const int other = (axis == 1) ? pl->nz : pl->ny;
    const int pmin = (sizeof(T) == 4) ? 2 : 1;
    const int pmax = 64 / (int)sizeof(T);   // 128-byte row segments: wider tiles gained nothing
    P = env_int("ETD_PAIRS_STRIDED", 0);
    if (P <= 0) {
      P = maxp < pmax ? maxp : pmax;
      while (P > pmin && (pl->nx / (2 * P)) * (long long)other < 2 * pl->num_sms) P /= 2;
    }
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
  L.fn = k->fn;
  L.grid = dim3((unsigned)grid);
  L.block = dim3((unsigned)(P * k->tpp));
  L.smem = pass_smem_bytes(*k, P, two ? 2 : 1);
  L.kind = kind;
  memcpy(L.args, &a, sizeof(a));
  L.args_size = sizeof(a);
  L.alg_bytes = fields_rw * (double)pl->unknowns * sizeof(T);
  // One kernel serves every axis of a given length, with different tile sizes, so the opt-in
  // limit is raised to the device maximum (not to this launch's size, which a later launch of the
  // same kernel could then undercut).
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
  if (L.smem > (size_t)optin) return fail(ETD_ERR_UNSUPPORTED, "tile needs %zu B of shared memory (max %d)", L.smem, optin);
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
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

template <class T>
etd_status build_step(etd_plan_s* pl) {
  void** F = pl->F;
  enum { V = 0, N0 = 1, V2 = 2, PF = 3, N2 = 4 };
  pl->step.clear();
  Launch L;
  etd_status st;
#define ADD(op, axis, i0, i1, o0, o1, kind, rw)                                               \
  do {                                                                                         \
    st = make_launch<T>(pl, op, axis, i0, i1, o0, o1, kind, rw, L);                            \
    if (st != ETD_OK) return st;                                                               \
    pl->step.push_back(L);                                                                     \
  } while (0)
  if (pl->ndim == 2) {
    if (pl->scheme == 2) {
      ADD(OP_REACT, 0, F[V], nullptr, F[N0], nullptr, PK_REACT, 2);
      ADD(OP_S1, 1, F[V], F[N0], F[V2], F[PF], PK_S1, 4);
      ADD(OP_REACT, 0, F[V2], nullptr, F[N2], nullptr, PK_REACT, 2);
      ADD(OP_S2, 1, F[N2], F[PF], F[V], nullptr, PK_S2, 3);
    } else {
      ADD(OP_REACT, 0, F[V], nullptr, F[N0], nullptr, PK_REACT, 2);
      ADD(OP_RK1, 1, F[V], F[N0], F[V], nullptr, PK_RK1, 3);
    }
  } else {
    ADD(OP_TRANSFORM, 1, F[V], nullptr, F[V2], nullptr, PK_TRANSFORM, 2);
    ADD(OP_REACT, 0, F[V2], nullptr, F[N0], nullptr, PK_REACT, 2);
    ADD(OP_TRANSFORM, 1, F[N0], nullptr, F[N0], nullptr, PK_TRANSFORM, 2);
    if (pl->scheme == 2) {
      ADD(OP_S1, 2, F[V], F[N0], F[V2], F[PF], PK_S1, 4);
      ADD(OP_TRANSFORM, 1, F[V2], nullptr, F[V2], nullptr, PK_TRANSFORM, 2);
      ADD(OP_REACT, 0, F[V2], nullptr, F[N2], nullptr, PK_REACT, 2);
      ADD(OP_TRANSFORM, 1, F[N2], nullptr, F[N2], nullptr, PK_TRANSFORM, 2);
      ADD(OP_S2, 2, F[N2], F[PF], F[V], nullptr, PK_S2, 3);
    } else {
      ADD(OP_RK1, 2, F[V], F[N0], F[V], nullptr, PK_RK1, 3);
    }
  }
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

etd_status entry_exit_any(etd_plan_s* pl, bool entry, void* u, std::vector<Launch>& out) {
  return pl->elem == 4 ? entry_exit<float>(pl, entry, u, out) : entry_exit<double>(pl, entry, u, out);
}

template <class T>
etd_status upload_tables(etd_plan_s* pl) {
  // FP64 on the host, rounded once to T: per axis tw (2M, M = FFT length), sn, zeta, ex, ec (N each)
  int fftM[3] = {0, 0, 0};
  const KernelInfo* kinf[3] = {nullptr, nullptr, nullptr};
  size_t total = 0;
  for (int a = 0; a < pl->ndim; ++a) {
    const KernelInfo* k = find_pass_kernel((int)sizeof(T), (int)pl->N[a], pl->odd[a]);
    if (!k) return fail(ETD_ERR_UNSUPPORTED, "no kernel for axis length %lld", (long long)pl->N[a]);
    fftM[a] = k->fft_len;
    kinf[a] = k;
    total += 2 * (size_t)(k->twn > 0 ? k->twn : 1) + 4 * (size_t)pl->N[a];
  }
  std::vector<T> h(total);
  size_t off = 0;
  size_t offs[3][5];
  for (int a = 0; a < pl->ndim; ++a) {
    const int n = (int)pl->N[a];
    const double hh = pl->h[a];
    // per-pass twiddle tables: pass with NS > 1 and radix R holds exp(2 pi i k r / (NS R)) at
    // [(r-1)*NS + k], k < NS, r = 1..R-1 (the layout the Stockham passes read)
    offs[a][0] = off;
    {
      size_t t = 0;
      int NS = 1;
      for (int i = 0; i < 4 && kinf[a]->radix[i]; ++i) {
        const int R = kinf[a]->radix[i];
        if (NS > 1) {
          for (int r = 1; r < R; ++r)
            for (int k = 0; k < NS; ++k, ++t) {
              const long long num = (long long)k * r % ((long long)NS * R);
              const double ang = 2.0 * M_PI * (double)num / (double)(NS * R);
              h[off + 2 * t] = (T)cos(ang);
              h[off + 2 * t + 1] = (T)sin(ang);
            }
        }
        NS *= R;
      }
      if (t == 0) {
        h[off] = T(1);
        h[off + 1] = T(0);
        t = 1;
      }
      off += 2 * t;
    }
    (void)fftM;
    offs[a][1] = off;
    for (int j = 0; j < n; ++j) h[off + j] = (T)sin(M_PI * (double)j / (double)n);
    off += n;
    offs[a][2] = off;
    offs[a][3] = off + n;
    offs[a][4] = off + 2 * n;
    for (int i = 0; i < n; ++i) {
      double zeta = 0.0;
      if (i > 0) {
        const double th = M_PI * (double)i / (double)n;
        const double s = sin(0.5 * th);
        const double mu = 12.0 / (hh * hh) * s * s / (2.0 + cos(th));  // (6/h^2)(1-cos)/(2+cos)
        zeta = pl->tau * pl->D * mu;
      }
      h[off + i] = (T)zeta;
      h[off + n + i] = (T)exp(-zeta);
      h[off + 2 * n + i] = (T)exp(-pl->opt.c2 * zeta);
    }
    off += 3 * (size_t)n;
    pl->sc[a] = 0.5 * sqrt(2.0 / (double)n);
  }
  ETD_CUDA(cudaMalloc(&pl->tables, total * sizeof(T)));
  ETD_CUDA(cudaMemcpy(pl->tables, h.data(), total * sizeof(T), cudaMemcpyHostToDevice));
  T* base = static_cast<T*>(pl->tables);
  for (int a = 0; a < pl->ndim; ++a) {
    pl->tw[a] = base + offs[a][0];
    pl->sn[a] = base + offs[a][1];
    pl->zeta[a] = base + offs[a][2];
    pl->ex[a] = base + offs[a][3];
    pl->ec[a] = base + offs[a][4];
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

}  // namespace

extern "C" {

etd_status etd_options_default(etd_options* opt) {
  if (!opt) return fail(ETD_ERR_INVALID_ARG, "opt is NULL");
  opt->dtype = ETD_F64;
  opt->route = ETD_ROUTE_AUTO;
  opt->c2 = 0.5;
  opt->flin = 1.0;
  opt->fcub = -1.0;
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
  if (!std::isfinite(o.flin) || !std::isfinite(o.fcub)) return fail(ETD_ERR_INVALID_ARG, "reaction coefficients must be finite");
  if (o.dtype != ETD_F32 && o.dtype != ETD_F64) return fail(ETD_ERR_INVALID_ARG, "dtype must be ETD_F32 or ETD_F64");
  if (o.route != ETD_ROUTE_AUTO && o.route != ETD_ROUTE_FFT && o.route != ETD_ROUTE_FFT_HALF)
    return fail(ETD_ERR_INVALID_ARG, "unknown route");
  for (int a = 0; a < ndim; ++a) {
    if (N[a] < 2) return fail(ETD_ERR_INVALID_ARG, "N[%d] = %lld < 2", a, (long long)N[a]);
    if (N[a] % 2) return fail(ETD_ERR_INVALID_ARG, "N[%d] = %lld must be even", a, (long long)N[a]);
    if (!(std::isfinite(h[a]) && h[a] > 0)) return fail(ETD_ERR_INVALID_ARG, "h[%d] must be finite and > 0", a);
  }
  for (int a = 0; a < ndim; ++a)
    if (!supported_length(N[a]))
      return fail(ETD_ERR_UNSUPPORTED, "N[%d] = %lld: supported lengths are 2^k (4..2048) and 3*2^k (6..1536)", a,
                  (long long)N[a]);
  etd_plan_s* pl = new etd_plan_s();
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
    if (o.dtype != ETD_F32 || o.route == ETD_ROUTE_FFT_HALF) pl->odd[a] = 0;
    else if (o.route == ETD_ROUTE_FFT) pl->odd[a] = 1;
    else pl->odd[a] = N[a] >= 512 ? 1 : 0;
  }
  pl->nx = (int)N[0];
  pl->ny = (int)N[1];
  pl->nz = ndim == 3 ? (int)N[2] : 1;
  pl->nfield = (size_t)pl->nx * pl->ny * pl->nz;
  pl->unknowns = (N[0] - 1) * (N[1] - 1) * (ndim == 3 ? N[2] - 1 : 1);
  auto bail = [&](etd_status s) {
    etd_destroy(pl);
    return s;
  };
  if (cudaGetDevice(&pl->device) != cudaSuccess) return bail(fail(ETD_ERR_CUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
  const size_t fbytes = pl->nfield * pl->elem;
  pl->ws_bytes = 5 * fbytes;
  cudaError_t e = cudaMalloc(&pl->ws, pl->ws_bytes);
  if (e != cudaSuccess) return bail(fail(ETD_ERR_OOM, "workspace of %zu bytes: %s", pl->ws_bytes, cudaGetErrorString(e)));
  e = cudaMemset(pl->ws, 0, pl->ws_bytes);
  if (e != cudaSuccess) return bail(fail(ETD_ERR_CUDA, "memset: %s", cudaGetErrorString(e)));
  for (int f = 0; f < 5; ++f) pl->F[f] = static_cast<char*>(pl->ws) + f * fbytes;
  etd_status st = (pl->elem == 4) ? upload_tables<float>(pl) : upload_tables<double>(pl);
  if (st != ETD_OK) return bail(st);
  st = (pl->elem == 4) ? build_step<float>(pl) : build_step<double>(pl);
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

etd_status etd_run(etd_plan pl, void* u, int64_t nsteps, void* stream) {
  if (!pl || !u) return fail(ETD_ERR_INVALID_ARG, "plan or u is NULL");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  if (nsteps == 0) return ETD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<Launch> ent, ext;
  etd_status st = entry_exit_any(pl, true, u, ent);
  if (st != ETD_OK) return st;
  st = entry_exit_any(pl, false, u, ext);
  if (st != ETD_OK) return st;
  for (const Launch& L : ent)
    if ((st = launch(L, s)) != ETD_OK) return st;
  if ((st = run_steps(pl, nsteps, s)) != ETD_OK) return st;
  for (const Launch& L : ext)
    if ((st = launch(L, s)) != ETD_OK) return st;
  return ETD_OK;
}

etd_status etd_step(etd_plan pl, void* u, void* stream) { return etd_run(pl, u, 1, stream); }

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
  return ETD_OK;
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
    g.m[a] = a < pl->ndim ? (int)pl->N[a] - 1 : 1;
    g.h[a] = a < pl->ndim ? pl->h[a] : 1.0;
  }
  g.D = pl->D;
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
  if (bad) return fail(ETD_ERR_NONFINITE, "%lld non-finite values", bad);
  return ETD_OK;
}

etd_status etd_run_profiled(etd_plan pl, void* u, int64_t nsteps, void* stream, double* ms, int64_t* cnt) {
  if (!pl || !u || !ms || !cnt) return fail(ETD_ERR_INVALID_ARG, "NULL argument");
  if (nsteps < 0) return fail(ETD_ERR_INVALID_ARG, "nsteps < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < ETD_NUM_PASS_KINDS; ++k) {
    ms[k] = 0;
    cnt[k] = 0;
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
  if (pl->host_dev) cudaFree(pl->host_dev);
  if (pl->mon_part) cudaFree(pl->mon_part);
  delete pl;
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
  }
  return "unknown status";
}

const char* etd_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
