// sno.cu - spectral neural operator (forward, gradient, Adam) and the Parareal driver, declared in
// include/etd_sno.h. All arithmetic runs in the kernels of sno_kernels.cuh; this file sizes the
// buffers, expresses every contraction as a strided batched GEMM and sequences the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/etd.h"
#include "../../include/etd_sno.h"
#include "sno_kernels.cuh"
#include "sno_mma.cuh"

void etd_internal_set_error(const char* msg);   // etd_api.cu

using namespace etd::sno;

namespace {

etd_status sfail(etd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  etd_internal_set_error(buf);
  return s;
}

#define SNO_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return sfail(e_ == cudaErrorMemoryAllocation ? ETD_ERR_OOM : ETD_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                   cudaGetErrorString(e_), __FILE__, __LINE__);                                     \
  } while (0)

int grid_for(long long n, int per = 256) {
  long long g = (n + per - 1) / per;
  if (g > 65536) g = 65536;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

struct etd_sno_s {
  int N = 0, n = 0, C = 0, M = 0, L = 0, Bmax = 0;
  long long npix = 0;
  // parameter layout offsets (floats)
  long long oWl = 0, obl = 0, oWm = 0, oWp = 0, obp = 0, oWq = 0, obq = 0, nparam = 0;
  float* W = nullptr;      // parameters
  float* G = nullptr;      // gradient
  float* Mo = nullptr;     // Adam first moment
  float* Ve = nullptr;     // Adam second moment
  int adam_t = 0;
  float* S = nullptr;      // S_M [M][n]
  float* a = nullptr;      // feature per field [Bmax]
  float* ahost = nullptr;  // pinned staging for a
  std::vector<float*> h;   // h_0..h_L [Bmax][C][npix]
  std::vector<float*> z;   // z_0..z_{L-1}
  std::vector<float*> hh;  // [Bmax][C][M][M]
  float* T = nullptr;      // transform scratch [Bmax][C][n][M] (also [M][n])
  float* gh = nullptr;     // [Bmax][C][M][M]
  float* dgh = nullptr;
  float* dh0 = nullptr;    // gradient ping-pong [Bmax][C][npix]
  float* dh1 = nullptr;
  float* uhat = nullptr;   // [Bmax][npix] (training)
  float* du = nullptr;     // [Bmax][npix]
  float* part = nullptr;   // reduction partials
  long long part_len = 0;
  double* lpart = nullptr; // loss partials
  int lblocks = 0;
  // forward contractions on the tensor cores (BF16 operands, FP32 accumulation) when every K and output
  // width fits a tile (n, C <= 256); the backward keeps FP32 (the exact straight-through gradient)
  bool tc = false;
  int num_sms = 148;
  int* err = nullptr;      // set by a tensor-core kernel whose wait ran out
};

namespace {

// ---- strided batched GEMM launcher
struct GemmOp {
  SGemm g;
  GemmOp(int M, int N, int K, int batch) {
    memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = N;
    g.K = K;
    g.batch = batch;
    g.alpha = 1.f;
    g.ksplit = 1;
  }
  GemmOp& A(const float* p, long long rs, long long cs, long long bs) {
    g.A = p; g.a_rs = rs; g.a_cs = cs; g.a_bs = bs;
    return *this;
  }
  GemmOp& B(const float* p, long long rs, long long cs, long long bs) {
    g.B = p; g.b_rs = rs; g.b_cs = cs; g.b_bs = bs;
    return *this;
  }
  GemmOp& Cm(float* p, long long rs, long long cs, long long bs) {
    g.C = p; g.c_rs = rs; g.c_cs = cs; g.c_bs = bs;
    return *this;
  }
  template <int BM, int BN>
  etd_status launch(cudaStream_t s) const {
    const int ks = g.ksplit > 1 ? g.ksplit : 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch * ks);
    if (grid.z > 65535u) return sfail(ETD_ERR_UNSUPPORTED, "GEMM batch %u too large", grid.z);
    sgemm_kernel<BM, BN><<<grid, 256, 0, s>>>(g);
    SNO_CUDA(cudaGetLastError());
    return ETD_OK;
  }
  // tile shape by output shape: skinny outputs get skinny tiles, large ones 128 x 128
  etd_status run(cudaStream_t s) const {
    if (g.M <= 32) return launch<32, 128>(s);
    if (g.N <= 32) return launch<128, 32>(s);
    if (g.M >= 128 && g.N >= 128) return launch<128, 128>(s);
    return launch<64, 64>(s);
  }
};

// ---- tensor-core contractions (sno_mma.cuh): NCOL >= the output columns, K <= 256
template <int NCOL, int EPI>
etd_status mma_launch(const MmaArgs& g, int num_sms, cudaStream_t s) {
  const size_t smem = mma_smem_bytes(NCOL, g.kpad);
  static bool attr_set = false;   // one kernel per (NCOL, EPI); the largest size any call can ask for
  if (!attr_set) {
    SNO_CUDA(cudaFuncSetAttribute(sno_mma_kernel<NCOL, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024));
    attr_set = true;
  }
  // CTAs per SM: at most 512 / NCOL (tensor-memory columns; a CTA that cannot allocate would wait for
  // a co-resident one to finish), at most 2048 / kMmaThreads (threads); where the columns are the
  // tighter limit the launch asks for enough shared memory that no more CTAs fit. The grid covers
  // that many per SM (CTAs loop over tiles).
  const int by_threads = 2048 / kMmaThreads;
  const int per_sm = std::min(by_threads, 512 / NCOL);
  const size_t floor_bytes = (size_t)228 * 1024 / (per_sm + 1) + 1024;
  const size_t launch_smem = std::max(smem, per_sm < by_threads ? floor_bytes : (size_t)0);
  const long long tiles = (long long)g.tiles_per_img * g.imgs;
  const int fit = (int)std::min<size_t>(per_sm, (size_t)227 * 1024 / launch_smem);
  const int grid = (int)std::min<long long>(tiles, (long long)std::max(1, fit) * num_sms);
  sno_mma_kernel<NCOL, EPI><<<grid, kMmaThreads, launch_smem, s>>>(g);
  SNO_CUDA(cudaGetLastError());
  return ETD_OK;
}
template <int EPI>
etd_status mma_run(const MmaArgs& g, int num_sms, cudaStream_t s) {
  if (g.ncol <= 32) return mma_launch<32, EPI>(g, num_sms, s);
  if (g.ncol <= 64) return mma_launch<64, EPI>(g, num_sms, s);
  if (g.ncol <= 128) return mma_launch<128, EPI>(g, num_sms, s);
  return mma_launch<256, EPI>(g, num_sms, s);
}

#define SNO_TRY(x)                     \
  do {                                 \
    etd_status st_ = (x);              \
    if (st_ != ETD_OK) return st_;     \
  } while (0)

// The dedicated kernel of the second truncated-transform contraction holds both M x n operands in
// shared memory.
bool small_modes(const etd_sno_s* m) { return m->M <= 32 && 2 * (size_t)m->M * m->n * sizeof(float) <= 227 * 1024; }

// out (M x M per image) = S_M X S_M^T for `imgs` images X (n x n); T is scratch (n x M per image).
// round: bf16-round the result. tc: the first contraction (X S_M^T, K = n) on the tensor cores with
// bf16 X and S_M, T then stored [M][n] per image.
etd_status modes_of(const etd_sno_s* m, const float* X, int imgs, float* out, bool round, bool tc, cudaStream_t s) {
  const int n = m->n, M = m->M;
  if (tc) {
    MmaArgs g;
    memset(&g, 0, sizeof(g));
    g.tiles_per_img = (n + 127) / 128;
    g.imgs = imgs;
    g.rows = n;
    g.kvalid = n;
    g.kpad = (n + 31) / 32 * 32;
    g.ncol = M;
    g.A = X;  g.a_rs = n;  g.a_ks = 1;  g.a_is = (long long)n * n;      // A[i][j] = X[i][j]
    g.B = m->S;  g.b_cs = n;  g.b_ks = 1;                               // B[m][j] = S_M[m][j]
    g.C = m->T;  g.c_rs = 1;  g.c_cs = n;  g.c_is = (long long)M * n;  // T[m][i]
    g.err = m->err;
    SNO_TRY(mma_run<ME_STORE>(g, m->num_sms, s));
    // out = S_M T^T  (M x M)
    if (small_modes(m)) {
      const size_t smem = 2 * (size_t)M * n * sizeof(float);
      static bool attr_set = false;
      if (!attr_set) {
        SNO_CUDA(cudaFuncSetAttribute(modes_pm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set = true;
      }
      modes_pm_kernel<<<imgs, 64, smem, s>>>(m->S, m->T, out, n, M, round ? 1 : 0);
      SNO_CUDA(cudaGetLastError());
      return ETD_OK;
    }
    GemmOp o(M, M, n, imgs);
    o.A(m->S, n, 1, 0).B(m->T, 1, n, (long long)M * n).Cm(out, M, 1, (long long)M * M);
    o.g.round_c = round ? 1 : 0;
    return o.run(s);
  }
  // T = X S_M^T  (n x M)
  SNO_TRY(GemmOp(n, M, n, imgs).A(X, n, 1, (long long)n * n).B(m->S, 1, n, 0).Cm(m->T, M, 1, (long long)n * M).run(s));
  // out = S_M T  (M x M)
  GemmOp o(M, M, n, imgs);
  o.A(m->S, n, 1, 0).B(m->T, M, 1, (long long)n * M).Cm(out, M, 1, (long long)M * M);
  o.g.round_c = round ? 1 : 0;
  return o.run(s);
}

// out (n x n per image) (+)= S_M^T Y S_M for `imgs` images Y (M x M); T is scratch (M x n per image).
// tc: the second contraction (S_M^T T, K = M) on the tensor cores with bf16 S_M and T.
etd_status field_of(const etd_sno_s* m, const float* Y, int imgs, float* out, float beta, bool tc, cudaStream_t s) {
  const int n = m->n, M = m->M;
  // T = Y S_M  (M x n)
  if (M <= 32) {
    modes_to_rows_kernel<<<imgs, 256, 0, s>>>(Y, m->S, m->T, n, M);
    SNO_CUDA(cudaGetLastError());
  } else {
    SNO_TRY(GemmOp(M, n, M, imgs).A(Y, M, 1, (long long)M * M).B(m->S, n, 1, 0).Cm(m->T, n, 1, (long long)M * n).run(s));
  }
  if (tc) {
    // out[i][j] = sum_m S_M[m][i] T[m][j], as D[j][i] over tiles of 128 j
    MmaArgs g;
    memset(&g, 0, sizeof(g));
    g.tiles_per_img = (n + 127) / 128;
    g.imgs = imgs;
    g.rows = n;
    g.kvalid = M;
    g.kpad = (M + 31) / 32 * 32;
    g.ncol = n;
    g.A = m->T;  g.a_rs = 1;  g.a_ks = n;  g.a_is = (long long)M * n;  // A[j][m] = T[m][j]
    g.B = m->S;  g.b_cs = 1;  g.b_ks = n;                              // B[i][m] = S_M[m][i]
    g.C = out;  g.c_rs = 1;  g.c_cs = n;  g.c_is = (long long)n * n;   // out[i][j]
    g.beta = beta;
    g.err = m->err;
    return beta != 0.f ? mma_run<ME_ACCUM>(g, m->num_sms, s) : mma_run<ME_STORE>(g, m->num_sms, s);
  }
  // out = S_M^T T  (n x n)
  GemmOp o(n, n, M, imgs);
  o.A(m->S, 1, n, 0).B(m->T, n, 1, (long long)M * n).Cm(out, n, 1, (long long)n * n);
  o.g.beta = beta;
  return o.run(s);
}

// per-field feature a = (ln D - ln 1e-3) / ln 100, uploaded through pinned staging
etd_status upload_feature(etd_sno_s* m, const double* D, int B, cudaStream_t s) {
  SNO_CUDA(cudaStreamSynchronize(s));   // the staging buffer may still feed an earlier copy
  for (int b = 0; b < B; ++b) {
    if (!(std::isfinite(D[b]) && D[b] > 0)) return sfail(ETD_ERR_INVALID_ARG, "D[%d] must be finite and > 0", b);
    m->ahost[b] = (float)((std::log(D[b]) - std::log(1e-3)) / std::log(100.0));
  }
  SNO_CUDA(cudaMemcpyAsync(m->a, m->ahost, B * sizeof(float), cudaMemcpyHostToDevice, s));
  return ETD_OK;
}

}  // namespace

namespace {

void sno_free(etd_sno_s* m) {
  float* bufs[] = {m->W, m->G, m->Mo, m->Ve, m->S, m->a, m->T, m->gh, m->dgh, m->dh0, m->dh1, m->uhat, m->du, m->part};
  for (float* p : bufs)
    if (p) cudaFree(p);
  for (float* p : m->h) cudaFree(p);
  for (float* p : m->z) cudaFree(p);
  for (float* p : m->hh) cudaFree(p);
  if (m->lpart) cudaFree(m->lpart);
  if (m->err) cudaFree(m->err);
  if (m->ahost) cudaFreeHost(m->ahost);
  delete m;
}

etd_status sno_alloc(float** p, long long count) {
  SNO_CUDA(cudaMalloc(p, (size_t)count * sizeof(float)));
  SNO_CUDA(cudaMemset(*p, 0, (size_t)count * sizeof(float)));
  return ETD_OK;
}

// Reads (and clears) the error word of the tensor-core kernels; call after synchronising.
etd_status check_err(etd_sno_s* m) {
  int e = 0;
  SNO_CUDA(cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    SNO_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return sfail(ETD_ERR_TIMEOUT, "a tensor-core contraction of the operator gave up waiting for its MMAs");
  }
  return ETD_OK;
}

// Forward pass for B fields; with `keep` it also keeps h, z, hh for the gradient (without, the
// pre-activations z are not stored: inference).
etd_status sno_forward(etd_sno_s* m, const float* u, int B, float* out, cudaStream_t s, bool keep) {
  const int C = m->C, M = m->M, L = m->L;
  const long long np = m->npix, img = (long long)C * np, M2 = (long long)M * M;
  lift_kernel<<<dim3(grid_for(np) < 64 ? grid_for(np) : 64, B * C), 256, 0, s>>>(u, m->a, m->W + m->oWl,
                                                                               m->W + m->obl, m->h[0], B, C, np);
  SNO_CUDA(cudaGetLastError());
  for (int l = 0; l < L; ++l) {
    SNO_TRY(modes_of(m, m->h[l], B * C, m->hh[l], true, m->tc, s));
    // gh[b][o][m] = sum_c bf(Wm[l][m][o][c]) hh[b][c][m], batched over modes m
    {
      GemmOp o(B, C, C, (int)M2);
      o.A(m->hh[l], C * M2, M2, 1).B(m->W + m->oWm + (long long)l * M2 * C * C, 1, C, (long long)C * C)
          .Cm(m->gh, C * M2, M2, 1);
      o.g.round_b = 1;
      SNO_TRY(o.run(s));
    }
    SNO_TRY(field_of(m, m->gh, B * C, m->z[l], 0.f, m->tc, s));
    // z[b] += Wp[l] h_l[b] + bp[l]; h_{l+1} = gelu(z)
    if (m->tc) {
      MmaArgs g;   // z[b][o][i] += sum_c bf(Wp[o][c]) bf(h[b][c][i]) + bp[o], as D[i][o] over tiles of 128 i
      memset(&g, 0, sizeof(g));
      g.tiles_per_img = (int)((np + 127) / 128);
      g.imgs = B;
      g.rows = (int)np;
      g.kvalid = C;
      g.kpad = (C + 31) / 32 * 32;
      g.ncol = C;
      g.A = m->h[l];  g.a_rs = 1;  g.a_ks = np;  g.a_is = img;
      g.B = m->W + m->oWp + (long long)l * C * C;  g.b_cs = C;  g.b_ks = 1;
      g.C = m->z[l];  g.c_rs = 1;  g.c_cs = np;  g.c_is = img;
      g.beta = 1.f;
      g.bias = m->W + m->obp + (long long)l * C;
      g.C2 = m->h[l + 1];
      g.err = m->err;
      SNO_TRY(keep ? mma_run<ME_PW_GELU>(g, m->num_sms, s) : mma_run<ME_PW_GELU_ONLY>(g, m->num_sms, s));
    } else {
      GemmOp o(C, (int)np, C, B);
      o.A(m->W + m->oWp + (long long)l * C * C, C, 1, 0).B(m->h[l], np, 1, img).Cm(m->z[l], np, 1, img);
      o.g.beta = 1.f;
      o.g.epi = SG_BIAS_GELU;
      o.g.bias = m->W + m->obp + (long long)l * C;
      o.g.C2 = m->h[l + 1];
      SNO_TRY(o.run(s));
    }
  }
  // out[b] = u[b] + Wq . h_L[b] + bq
  const int pblk = (int)std::min<long long>((np + 255) / 256, 64);
  project_kernel<<<dim3(pblk, B), 256, 0, s>>>(u, m->h[L], m->W + m->oWq, m->W + m->obq, out, C, np);
  SNO_CUDA(cudaGetLastError());
  return ETD_OK;
}

// sum over fields and pixels of X[b][c][i] * (y ? y[b][i] : 1), weighted per field by w (device,
// may be NULL), into G[off + c * stride] for c < C
etd_status chan_reduce(etd_sno_s* m, const float* X, const float* y, const float* w, int B, int C, long long off,
                       int stride, cudaStream_t s) {
  const int nblk = 16;
  if ((long long)B * C * nblk > m->part_len) return sfail(ETD_ERR_UNSUPPORTED, "reduction scratch too small");
  chan_dot_kernel<<<dim3(nblk, B * C), 256, 0, s>>>(X, y, C, m->npix, m->part);
  SNO_CUDA(cudaGetLastError());
  chan_combine_kernel<<<(C + 127) / 128, 128, 0, s>>>(m->part, nblk, w, B, C, m->G + off, stride, 0);
  SNO_CUDA(cudaGetLastError());
  return ETD_OK;
}

// Gradient of the loss; du holds d loss / d u_hat.
etd_status sno_backward(etd_sno_s* m, const float* u, int B, cudaStream_t s) {
  const int C = m->C, M = m->M, L = m->L;
  const long long np = m->npix, img = (long long)C * np, M2 = (long long)M * M;
  SNO_CUDA(cudaMemsetAsync(m->G, 0, (size_t)m->nparam * sizeof(float), s));
  // projection: dWq[c] = sum h_L[c] du, dbq = sum du, dh_L[b][c][i] = Wq[c] du[b][i]
  SNO_TRY(chan_reduce(m, m->h[L], m->du, nullptr, B, C, m->oWq, 1, s));
  SNO_TRY(chan_reduce(m, m->du, nullptr, nullptr, B, 1, m->obq, 1, s));
  float* dh = m->dh0;
  float* dn = m->dh1;
  SNO_TRY(GemmOp(C, (int)np, 1, B).A(m->W + m->oWq, 1, 0, 0).B(m->du, 0, 1, np).Cm(dh, np, 1, img).run(s));
  for (int l = L - 1; l >= 0; --l) {
    float* dz = m->z[l];   // overwritten: dz = dh * gelu'(z)
    gelu_backward_kernel<<<grid_for((long long)B * img), 256, 0, s>>>(dh, m->z[l], dz, (long long)B * img);
    SNO_CUDA(cudaGetLastError());
    SNO_TRY(chan_reduce(m, dz, nullptr, nullptr, B, C, m->obp + (long long)l * C, 1, s));
    // dWp[l][o][c] = sum_b sum_i dz[b][o][i] h_l[b][c][i]: per (field, K split) partials, then summed
    {
      const int ks = 16;
      if ((long long)B * ks * C * C > m->part_len) return sfail(ETD_ERR_UNSUPPORTED, "reduction scratch too small");
      GemmOp o(C, C, (int)np, B);
      o.A(dz, np, 1, img).B(m->h[l], 1, np, img).Cm(m->part, C, 1, (long long)ks * C * C);
      o.g.ksplit = ks;
      o.g.c_ss = (long long)C * C;
      SNO_TRY(o.run(s));
      reduce_batch_kernel<<<grid_for((long long)C * C), 256, 0, s>>>(m->part, m->G + m->oWp + (long long)l * C * C,
                                                                    B * ks, (long long)C * C, 0);
      SNO_CUDA(cudaGetLastError());
    }
    // spectral path: dgh = S_M dz S_M^T
    SNO_TRY(modes_of(m, dz, B * C, m->dgh, false, false, s));
    // dWm[l][m][o][c] = sum_b dgh[b][o][m] hh[b][c][m]
    SNO_TRY(GemmOp(C, C, B, (int)M2)
                .A(m->dgh, M2, C * M2, 1)
                .B(m->hh[l], C * M2, M2, 1)
                .Cm(m->G + m->oWm + (long long)l * M2 * C * C, C, 1, (long long)C * C)
                .run(s));
    // dhh[b][c][m] = sum_o bf(Wm[l][m][o][c]) dgh[b][o][m]   (into gh as scratch)
    {
      GemmOp o(B, C, C, (int)M2);
      o.A(m->dgh, C * M2, M2, 1).B(m->W + m->oWm + (long long)l * M2 * C * C, C, 1, (long long)C * C)
          .Cm(m->gh, C * M2, M2, 1);
      o.g.round_b = 1;
      SNO_TRY(o.run(s));
    }
    // dh_l = Wp^T dz + S_M^T dhh S_M
    SNO_TRY(GemmOp(C, (int)np, C, B).A(m->W + m->oWp + (long long)l * C * C, 1, C, 0).B(dz, np, 1, img)
                .Cm(dn, np, 1, img).run(s));
    SNO_TRY(field_of(m, m->gh, B * C, dn, 1.f, false, s));
    float* t = dh;
    dh = dn;
    dn = t;
  }
  // lift: dWl[c][0] = sum dh0 u, dWl[c][1] = sum_b a[b] sum_i dh0, dbl[c] = sum dh0
  SNO_TRY(chan_reduce(m, dh, u, nullptr, B, C, m->oWl, 2, s));
  SNO_TRY(chan_reduce(m, dh, nullptr, m->a, B, C, m->oWl + 1, 2, s));
  SNO_TRY(chan_reduce(m, dh, nullptr, nullptr, B, C, m->obl, 1, s));
  return ETD_OK;
}

}  // namespace

extern "C" {

etd_status etd_sno_create(etd_sno* out, int N, int C, int M, int L, int max_batch) {
  etd_internal_set_error("");
  if (!out) return sfail(ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 8 || N > 2048 || N % 2) return sfail(ETD_ERR_INVALID_ARG, "N must be even, 8..2048");
  if (C < 1 || C > 256) return sfail(ETD_ERR_INVALID_ARG, "C must be 1..256");
  if (M < 1 || M >= N) return sfail(ETD_ERR_INVALID_ARG, "M must be 1..N-1");
  if (L < 1 || L > 16) return sfail(ETD_ERR_INVALID_ARG, "L must be 1..16");
  if (max_batch < 1 || (long long)max_batch * C > 65535) return sfail(ETD_ERR_INVALID_ARG, "max_batch * C must be 1..65535");
  etd_sno_s* m = new etd_sno_s();
  m->N = N;
  m->n = N - 1;
  m->C = C;
  m->M = M;
  m->L = L;
  m->Bmax = max_batch;
  m->npix = (long long)m->n * m->n;
  const long long M2 = (long long)M * M;
  m->oWl = 0;
  m->obl = m->oWl + 2LL * C;
  m->oWm = m->obl + C;
  m->oWp = m->oWm + (long long)L * M2 * C * C;
  m->obp = m->oWp + (long long)L * C * C;
  m->oWq = m->obp + (long long)L * C;
  m->obq = m->oWq + C;
  m->nparam = m->obq + 1;
  auto bail = [&](etd_status st) {
    sno_free(m);
    return st;
  };
  const long long act = (long long)max_batch * C * m->npix;
  etd_status st;
  if ((st = sno_alloc(&m->W, m->nparam)) != ETD_OK || (st = sno_alloc(&m->G, m->nparam)) != ETD_OK ||
      (st = sno_alloc(&m->Mo, m->nparam)) != ETD_OK || (st = sno_alloc(&m->Ve, m->nparam)) != ETD_OK ||
      (st = sno_alloc(&m->S, (long long)M * m->n)) != ETD_OK || (st = sno_alloc(&m->a, max_batch)) != ETD_OK ||
      (st = sno_alloc(&m->T, (long long)max_batch * C * m->n * M)) != ETD_OK ||
      (st = sno_alloc(&m->gh, (long long)max_batch * C * M2)) != ETD_OK ||
      (st = sno_alloc(&m->dgh, (long long)max_batch * C * M2)) != ETD_OK ||
      (st = sno_alloc(&m->dh0, act)) != ETD_OK || (st = sno_alloc(&m->dh1, act)) != ETD_OK ||
      (st = sno_alloc(&m->uhat, (long long)max_batch * m->npix)) != ETD_OK ||
      (st = sno_alloc(&m->du, (long long)max_batch * m->npix)) != ETD_OK)
    return bail(st);
  m->part_len = std::max((long long)max_batch * C * 16, (long long)max_batch * 16 * C * C);
  if ((st = sno_alloc(&m->part, m->part_len)) != ETD_OK) return bail(st);
  for (int l = 0; l <= L; ++l) {
    float* p = nullptr;
    if ((st = sno_alloc(&p, act)) != ETD_OK) return bail(st);
    m->h.push_back(p);
    if (l < L) {
      if ((st = sno_alloc(&p, act)) != ETD_OK) return bail(st);
      m->z.push_back(p);
      if ((st = sno_alloc(&p, (long long)max_batch * C * M2)) != ETD_OK) return bail(st);
      m->hh.push_back(p);
    }
  }
  m->lblocks = 512;
  if (cudaMalloc(&m->lpart, m->lblocks * sizeof(double)) != cudaSuccess) return bail(sfail(ETD_ERR_OOM, "loss scratch"));
  if (cudaMallocHost(&m->ahost, max_batch * sizeof(float)) != cudaSuccess) return bail(sfail(ETD_ERR_OOM, "pinned staging"));
  // S_M[p][j] = sqrt(2/N) sin(pi ((p+1)(j+1) mod 2N) / N), FP64 on the host
  std::vector<float> hs((size_t)M * m->n);
  for (int p = 0; p < M; ++p)
    for (int j = 0; j < m->n; ++j)
      hs[(size_t)p * m->n + j] =
          (float)(std::sqrt(2.0 / N) * std::sin(M_PI * (double)(((long long)(p + 1) * (j + 1)) % (2LL * N)) / N));
  if (cudaMemcpy(m->S, hs.data(), hs.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(sfail(ETD_ERR_CUDA, "upload of the mode matrix"));
  m->tc = m->n <= 256 && C <= 256 && M <= 256;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&m->err, sizeof(int)) != cudaSuccess || cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess)
    return bail(sfail(ETD_ERR_OOM, "error word"));
  *out = m;
  return ETD_OK;
}

int64_t etd_sno_param_count(etd_sno m) { return m ? m->nparam : 0; }

etd_status etd_sno_set_params(etd_sno m, const float* host) {
  if (!m || !host) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  SNO_CUDA(cudaMemcpy(m->W, host, (size_t)m->nparam * sizeof(float), cudaMemcpyHostToDevice));
  SNO_CUDA(cudaMemset(m->Mo, 0, (size_t)m->nparam * sizeof(float)));
  SNO_CUDA(cudaMemset(m->Ve, 0, (size_t)m->nparam * sizeof(float)));
  m->adam_t = 0;
  return ETD_OK;
}

etd_status etd_sno_get_params(etd_sno m, float* host) {
  if (!m || !host) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  SNO_CUDA(cudaDeviceSynchronize());
  SNO_CUDA(cudaMemcpy(host, m->W, (size_t)m->nparam * sizeof(float), cudaMemcpyDeviceToHost));
  return ETD_OK;
}

etd_status etd_sno_forward(etd_sno m, const float* u, const double* D, int B, float* out, void* stream) {
  if (!m || !u || !D || !out) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  if (B < 1 || B > m->Bmax) return sfail(ETD_ERR_INVALID_ARG, "B = %d outside 1..%d", B, m->Bmax);
  if (out == u) return sfail(ETD_ERR_INVALID_ARG, "out may not alias u");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SNO_TRY(upload_feature(m, D, B, s));
  return sno_forward(m, u, B, out, s, false);
}

etd_status etd_sno_train_step(etd_sno m, const float* u, const double* D, const float* target, int B, float lr,
                              double* loss, float* grads_out, void* stream) {
  if (!m || !u || !D || !target) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  if (B < 1 || B > m->Bmax) return sfail(ETD_ERR_INVALID_ARG, "B = %d outside 1..%d", B, m->Bmax);
  if (!(std::isfinite(lr) && lr >= 0)) return sfail(ETD_ERR_INVALID_ARG, "lr must be finite and >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SNO_TRY(upload_feature(m, D, B, s));
  SNO_TRY(sno_forward(m, u, B, m->uhat, s, true));
  const long long n = (long long)B * m->npix;
  mse_grad_kernel<<<m->lblocks, 256, 0, s>>>(m->uhat, target, m->du, n, m->lpart);
  SNO_CUDA(cudaGetLastError());
  SNO_TRY(sno_backward(m, u, B, s));
  if (grads_out) {
    SNO_CUDA(cudaMemcpyAsync(grads_out, m->G, (size_t)m->nparam * sizeof(float), cudaMemcpyDeviceToHost, s));
  } else {
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, m->adam_t)), c2 = (float)(1.0 - std::pow(0.999, m->adam_t));
    adam_kernel<<<grid_for(m->nparam), 256, 0, s>>>(m->W, m->G, m->Mo, m->Ve, m->nparam, lr, b1, b2, 1e-8f, c1, c2);
    SNO_CUDA(cudaGetLastError());
  }
  std::vector<double> lp(m->lblocks);
  SNO_CUDA(cudaMemcpyAsync(lp.data(), m->lpart, m->lblocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  SNO_CUDA(cudaStreamSynchronize(s));
  SNO_TRY(check_err(m));
  if (loss) {
    double t = 0.0;
    for (double v : lp) t += v;
    *loss = t / (double)n;
  }
  return ETD_OK;
}

etd_status etd_sno_destroy(etd_sno m) {
  if (m) sno_free(m);
  return ETD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Parareal with the SNO (or one long ETDRK2 step) as coarse and batched ETDRK2 as fine propagator.

struct etd_parareal_s {
  etd_sno sno = nullptr;
  int N = 0, B = 0, W = 0, steps = 0;
  long long npix = 0;
  double tau = 0;
  std::vector<double> D;
  // fine[k]: the windows k .. W-1 of every problem, (W - k) * B problems (window n of problem b at
  // (n - k) * B + b); an iteration propagates only the windows not yet converged
  std::vector<etd_batch> fine;
  etd_batch fine_one = nullptr;   // B problems (fallback)
  etd_batch coarse = nullptr;     // B problems, one step of steps * tau (no SNO)
  float* U = nullptr;             // (W + 1) * B fields: current iterate
  float* V = nullptr;             // (W + 1) * B fields: next iterate
  float* F = nullptr;             // W * B fields
  float* Go = nullptr;            // W * B fields: coarse values of the current iterate
  float* Gn = nullptr;            // B fields
  double* part = nullptr;         // norm partials [B][nblk][2]
  int nblk = 32;
  std::vector<void*> ptr_all, ptr_one;
};

namespace {

etd_status make_batch(etd_batch* out, int count, int N, const double* D, int Dcount, double tau) {
  std::vector<int64_t> Ns(2 * (size_t)count, N);
  std::vector<double> hs(2 * (size_t)count, 1.0 / N), Ds(count);
  for (int i = 0; i < count; ++i) Ds[i] = D[i % Dcount];
  etd_options o;
  etd_options_default(&o);
  o.dtype = ETD_F32;
  return etd_batch_create(out, count, Ns.data(), hs.data(), Ds.data(), tau, ETD_ETDRK2, &o);
}

// one coarse application for the B fields at `in`, into `out`
etd_status coarse_apply(etd_parareal_s* p, const float* in, float* out, cudaStream_t s) {
  if (p->sno) return etd_sno_forward(p->sno, in, p->D.data(), p->B, out, s);
  SNO_CUDA(cudaMemcpyAsync(out, in, (size_t)p->B * p->npix * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int b = 0; b < p->B; ++b) p->ptr_one[b] = out + (size_t)b * p->npix;
  return etd_batch_run(p->coarse, p->ptr_one.data(), 1, s);
}

// the fine propagator on the B fields at `in`, into `out`
etd_status fine_one(etd_parareal_s* p, const float* in, float* out, cudaStream_t s) {
  SNO_CUDA(cudaMemcpyAsync(out, in, (size_t)p->B * p->npix * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int b = 0; b < p->B; ++b) p->ptr_one[b] = out + (size_t)b * p->npix;
  return etd_batch_run(p->fine_one, p->ptr_one.data(), p->steps, s);
}

}  // namespace

extern "C" {

etd_status etd_parareal_create(etd_parareal* out, etd_sno sno, int N, int B, const double* D, double tau,
                               int window_steps, int windows) {
  if (!out || !D) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (B < 1 || windows < 1 || windows > 32 || window_steps < 1) return sfail(ETD_ERR_INVALID_ARG, "bad sizes");
  if (!(std::isfinite(tau) && tau > 0)) return sfail(ETD_ERR_INVALID_ARG, "tau must be finite and > 0");
  if (sno && (sno->N != N || B > sno->Bmax)) return sfail(ETD_ERR_INVALID_ARG, "the SNO's mesh or batch does not fit");
  etd_parareal_s* p = new etd_parareal_s();
  p->sno = sno;
  p->N = N;
  p->B = B;
  p->W = windows;
  p->steps = window_steps;
  p->tau = tau;
  p->npix = (long long)(N - 1) * (N - 1);
  p->D.assign(D, D + B);
  auto bail = [&](etd_status st) {
    etd_parareal_destroy(p);
    return st;
  };
  etd_status st;
  p->fine.assign(windows, nullptr);
  for (int k = 0; k < windows; ++k)
    if ((st = make_batch(&p->fine[k], (windows - k) * B, N, D, B, tau)) != ETD_OK) return bail(st);
  if ((st = make_batch(&p->fine_one, B, N, D, B, tau)) != ETD_OK) return bail(st);
  if (!sno && (st = make_batch(&p->coarse, B, N, D, B, tau * window_steps)) != ETD_OK) return bail(st);
  const size_t fb = (size_t)B * p->npix * sizeof(float);
  if (cudaMalloc(&p->U, (windows + 1) * fb) != cudaSuccess || cudaMalloc(&p->V, (windows + 1) * fb) != cudaSuccess ||
      cudaMalloc(&p->F, windows * fb) != cudaSuccess || cudaMalloc(&p->Go, windows * fb) != cudaSuccess ||
      cudaMalloc(&p->Gn, fb) != cudaSuccess ||
      cudaMalloc(&p->part, (size_t)B * p->nblk * 2 * sizeof(double)) != cudaSuccess)
    return bail(sfail(ETD_ERR_OOM, "Parareal states"));
  p->ptr_all.resize((size_t)windows * B);
  p->ptr_one.resize(B);
  *out = p;
  return ETD_OK;
}

etd_status etd_parareal_run(etd_parareal p, const float* u0, float* u_out, int max_iter, double tol,
                            double fallback_tol, etd_parareal_stats* stats, void* stream) {
  if (!p || !u0 || !u_out) return sfail(ETD_ERR_INVALID_ARG, "NULL argument");
  if (max_iter < 0 || max_iter > 32) return sfail(ETD_ERR_INVALID_ARG, "max_iter must be 0..32");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int B = p->B, W = p->W;
  const size_t fe = (size_t)B * p->npix;   // floats per window state
  etd_parareal_stats st{};
  auto win = [&](float* base, int n) { return base + (size_t)n * fe; };
  // coarse sweep U^0
  SNO_CUDA(cudaMemcpyAsync(p->U, u0, fe * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int n = 0; n < W; ++n) {
    SNO_TRY(coarse_apply(p, win(p->U, n), win(p->Go, n), s));
    SNO_CUDA(cudaMemcpyAsync(win(p->U, n + 1), win(p->Go, n), fe * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  std::vector<double> hp((size_t)B * p->nblk * 2);
  // U_0 .. U_d are the fine solution itself: U_0 = u0, and each iteration makes at least one more window
  // exact (the window after the exact prefix takes F of an exact start; a fallback from an exact start
  // extends the prefix too). Those windows keep their values: in exact arithmetic the Parareal update
  // gives them F(U_n) anyway, and recomputing G(U_n^{k+1}) - G(U_n^k) there would only add the coarse
  // propagator's rounding (bf16 in the operator, not Lipschitz in its input) to converged states.
  int d = 0;
  for (int k = 1; k <= max_iter && d < W; ++k) {
    // fine propagation of the windows d .. W-1 of the current iterate (the earlier ones are converged), in
    // one batched run
    SNO_CUDA(cudaMemcpyAsync(win(p->F, d), win(p->U, d), (size_t)(W - d) * fe * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < (W - d) * B; ++i) p->ptr_all[i] = win(p->F, d) + (size_t)i * p->npix;
    SNO_TRY(etd_batch_run(p->fine[d], p->ptr_all.data(), p->steps, s));
    // sequential correction sweep
    SNO_CUDA(cudaMemcpyAsync(p->V, p->U, (size_t)(d + 1) * fe * sizeof(float), cudaMemcpyDeviceToDevice, s));
    double worst = 0.0;
    int dn = d;
    for (int n = d; n < W; ++n) {
      const bool exact_start = n == d;   // U_n = V_n is the fine solution: V_{n+1} = F(U_n)
      if (!exact_start) SNO_TRY(coarse_apply(p, win(p->V, n), p->Gn, s));
      parareal_update_kernel<<<dim3(p->nblk, B), 256, 0, s>>>(exact_start ? nullptr : p->Gn, win(p->F, n),
                                                             win(p->Go, n), win(p->U, n + 1), win(p->V, n + 1),
                                                             p->npix, p->part);
      SNO_CUDA(cudaGetLastError());
      if (!exact_start)
        SNO_CUDA(cudaMemcpyAsync(win(p->Go, n), p->Gn, fe * sizeof(float), cudaMemcpyDeviceToDevice, s));
      SNO_CUDA(cudaMemcpyAsync(hp.data(), p->part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      SNO_CUDA(cudaStreamSynchronize(s));
      double corr = 0.0;
      for (int b = 0; b < B; ++b) {
        double a = 0.0, e2 = 0.0;
        for (int j = 0; j < p->nblk; ++j) {
          a += hp[((size_t)b * p->nblk + j) * 2];
          e2 += hp[((size_t)b * p->nblk + j) * 2 + 1];
        }
        corr = std::max(corr, a > 0 ? std::sqrt(e2 / a) : std::sqrt(e2));
      }
      if (exact_start) {
        dn = n + 1;
      } else if (k > 1 && corr > fallback_tol) {   // rejected: advance this window with the plain solver
        SNO_TRY(fine_one(p, win(p->V, n), win(p->V, n + 1), s));
        st.fallbacks += 1;
        if (dn == n) dn = n + 1;
      }
      worst = std::max(worst, corr);
    }
    std::swap(p->U, p->V);
    d = dn;
    st.iterations = k;
    st.correction[k - 1] = worst;
    if (worst < tol) break;
  }
  SNO_CUDA(cudaMemcpyAsync(u_out, win(p->U, W), fe * sizeof(float), cudaMemcpyDeviceToDevice, s));
  SNO_CUDA(cudaStreamSynchronize(s));
  if (p->sno) SNO_TRY(check_err(p->sno));
  if (stats) *stats = st;
  return ETD_OK;
}

etd_status etd_parareal_destroy(etd_parareal p) {
  if (!p) return ETD_OK;
  for (etd_batch f : p->fine)
    if (f) etd_batch_destroy(f);
  if (p->fine_one) etd_batch_destroy(p->fine_one);
  if (p->coarse) etd_batch_destroy(p->coarse);
  for (void* q : {(void*)p->U, (void*)p->V, (void*)p->F, (void*)p->Go, (void*)p->Gn, (void*)p->part})
    if (q) cudaFree(q);
  delete p;
  return ETD_OK;
}

}  // extern "C"
