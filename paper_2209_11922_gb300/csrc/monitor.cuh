// monitor.cuh - FP64 reductions over a dense nodal field: mass 1^T M U, energy, max|u|, #non-finite.
//
// M and K are the assembled Q1 matrices of eq. (4.1) (M = A_x (x) A_y [(x) A_z],
// K = D sum_a B_a (x) A_others), applied as their 3^d-point nodal stencils with zero Dirichlet
// values outside the interior (periodic: indices wrap around):
//   A_a: (h_a/6) [1 4 1],  B_a: (1/h_a) [-1 2 -1].
// The mass uses the column sums of A_a: (h_a/6)(4 + [i > 1] + [i < N_a - 1]) (periodic: h_a).
// energy = 1/2 U^T K U + sum_nodes prod(h) G(u), G(u) = (u^2 - 1)^2 / 4 when flog = 0, else the
// potential with G' = -f and G(0) = 0 of f = flin u + fcub u^3 + flog artanh u:
// G(u) = -flog (u artanh u + ln(1 - u^2)/2) - flin u^2/2 - fcub u^4/4 (the Flory-Huggins energy
// density of Example 5.3 for flin = theta_c, fcub = 0, flog = -theta).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace etd {

struct MonitorGeom {
  int ndim;
  int m[3];        // dense extents N_a - 1 (periodic: N_a; m[2] = 1 in 2D)
  double h[3];
  double D;
  int periodic;    // 1: stencils wrap around
  double flin, fcub, flog;   // reaction of the potential term (flog = 0: the double well)
};

template <class T>
__global__ void __launch_bounds__(256) monitor_partial_kernel(const T* __restrict__ u, MonitorGeom g,
                                                              double* __restrict__ part,
                                                              long long* __restrict__ nonfin) {
  const long long n = (long long)g.m[0] * g.m[1] * g.m[2];
  double s_mass = 0.0, s_quad = 0.0, s_pot = 0.0, s_max = 0.0;
  long long s_bad = 0;
  const double cell = g.h[0] * g.h[1] * (g.ndim == 3 ? g.h[2] : 1.0);
  double aw[3][3], bw[3][3];
  for (int a = 0; a < 3; ++a) {
    aw[a][0] = aw[a][2] = g.h[a] / 6.0;
    aw[a][1] = 4.0 * g.h[a] / 6.0;
    bw[a][0] = bw[a][2] = -1.0 / g.h[a];
    bw[a][1] = 2.0 / g.h[a];
  }
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.m[0]);
    const int j = (int)((idx / g.m[0]) % g.m[1]);
    const int k = (int)(idx / ((long long)g.m[0] * g.m[1]));
    const double v = (double)u[idx];
    if (!isfinite(v)) {
      ++s_bad;
      continue;
    }
    double w = 1.0;
    const int ii[3] = {i, j, k};
    for (int a = 0; a < g.ndim; ++a)
      w *= g.periodic ? g.h[a] : g.h[a] / 6.0 * (4.0 + (ii[a] > 0 ? 1.0 : 0.0) + (ii[a] < g.m[a] - 1 ? 1.0 : 0.0));
    s_mass += w * v;
    // (K U) at this node from the 3^d stencil
    double ku = 0.0;
    const int kz = g.ndim == 3 ? 1 : 0;
    // periodic axes wrap (their extents are >= 4, so the three stencil nodes are distinct)
    auto wrap = [&](int v, int n) { return g.periodic ? (v < 0 ? v + n : (v >= n ? v - n : v)) : v; };
    for (int dz = -kz; dz <= kz; ++dz) {
      const int zz = wrap(k + dz, g.m[2]);
      if (zz < 0 || zz >= g.m[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = wrap(j + dy, g.m[1]);
        if (yy < 0 || yy >= g.m[1]) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = wrap(i + dx, g.m[0]);
          if (xx < 0 || xx >= g.m[0]) continue;
          const double un = (double)u[((long long)zz * g.m[1] + yy) * g.m[0] + xx];
          const int d[3] = {dx + 1, dy + 1, dz + 1};
          double wk = 0.0;
          for (int a = 0; a < g.ndim; ++a) {
            double t = bw[a][d[a]];
            for (int b = 0; b < g.ndim; ++b)
              if (b != a) t *= aw[b][d[b]];
            wk += t;
          }
          ku += g.D * wk * un;
        }
      }
    }
    s_quad += 0.5 * v * ku;
    if (g.flog != 0.0)
      s_pot += cell * (-g.flog * (v * atanh(v) + 0.5 * log1p(-v * v)) - 0.5 * g.flin * v * v - 0.25 * g.fcub * v * v * v * v);
    else
      s_pot += cell * 0.25 * (v * v - 1.0) * (v * v - 1.0);
    s_max = fmax(s_max, fabs(v));
  }
  __shared__ double sh[4][256];
  __shared__ long long shb[256];
  const int t = threadIdx.x;
  sh[0][t] = s_mass;
  sh[1][t] = s_quad;
  sh[2][t] = s_pot;
  sh[3][t] = s_max;
  shb[t] = s_bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      sh[0][t] += sh[0][t + s];
      sh[1][t] += sh[1][t + s];
      sh[2][t] += sh[2][t + s];
      sh[3][t] = fmax(sh[3][t], sh[3][t + s]);
      shb[t] += shb[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    part[4 * blockIdx.x + 0] = sh[0][0];
    part[4 * blockIdx.x + 1] = sh[1][0];
    part[4 * blockIdx.x + 2] = sh[2][0];
    part[4 * blockIdx.x + 3] = sh[3][0];
    nonfin[blockIdx.x] = shb[0];
  }
}

// Reduces `nb` partial records into out[0..3] = mass, energy, maxabs and *bad (one block of 256).
// Internal linkage: every translation unit that launches it has its own copy.
static __global__ void __launch_bounds__(256) monitor_final_kernel(const double* __restrict__ part,
                                                            const long long* __restrict__ nonfin, int nb,
                                                            double* __restrict__ out, long long* __restrict__ bad) {
  __shared__ double sh[4][256];
  __shared__ long long shb[256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0, m = 0.0;
  long long k = 0;
  for (int i = t; i < nb; i += blockDim.x) {
    a += part[4 * i + 0];
    b += part[4 * i + 1];
    c += part[4 * i + 2];
    m = fmax(m, part[4 * i + 3]);
    k += nonfin[i];
  }
  sh[0][t] = a;
  sh[1][t] = b;
  sh[2][t] = c;
  sh[3][t] = m;
  shb[t] = k;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      sh[0][t] += sh[0][t + s];
      sh[1][t] += sh[1][t + s];
      sh[2][t] += sh[2][t + s];
      sh[3][t] = fmax(sh[3][t], sh[3][t + s]);
      shb[t] += shb[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0] + sh[2][0];
    out[2] = sh[3][0];
    *bad = shb[0];
  }
}

}  // namespace etd
