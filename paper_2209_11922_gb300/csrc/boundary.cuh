// boundary.cuh - nonhomogeneous Dirichlet data as part of f (Section 4; Example 5.2 of Section 5).
//
// The Galerkin system on all nodes with the boundary nodal values g(t) prescribed has the interior
// rows M_II U' + K_II U = M_II f(U) + b(t) with
//     b(t) = M_IB (f(g) - g'(t)) - K_IB g(t),
// so every stage adds M_II^{-1} b(t) to the nodal reaction. In the pitched state of a stage (spectral
// along every axis but the last) that term is S_last (Lambda_A^{-1} (.) S b) with S the product of the
// per-axis sine transforms and Lambda_A the tensor of mass eigenvalues, computed as
//     BUILD b -> DST along every axis -> SCALE by 1/(lambda^A_x lambda^A_y [lambda^A_z])
//             -> DST along the last axis -> ADD to the stage's reaction field,
// the transforms being the plan's own pass kernels. b is nonzero only on interior nodes next to the
// boundary; BUILD sums the 3^d-point Q1 stencils over their boundary neighbours:
//     M_ij = prod_a m_a(d_a),  K_ij = D sum_a k_a(d_a) prod_{b != a} m_b(d_b),
//     m(0) = 4h/6, m(+-1) = h/6, k(0) = 2/h, k(+-1) = -1/h,   d = j - i.
// Boundary values come from packed face arrays (x = 0, x = L_x, y = 0, y = L_y, z = 0, z = L_z, each
// over all its nodes, x fastest) with values then time derivatives, in FP64.
#pragma once
#include <cuda_runtime.h>

#include "etd_coeffs.cuh"

namespace etd {

template <class T> struct BndArgs {
  int ndim;
  int nx, ny, nz;          // pitched extents N_a (nz = 1 in 2D); node N_a is on the high face
  long long n;             // pitched entries nx * ny * nz
  T* out;                  // BUILD / SCALE: the B field; ADD: the stage's reaction field
  const T* in;             // ADD: the B field
  const double* g;         // BUILD: packed boundary values [count], then time derivatives [count]
  long long count;
  long long off[6];        // start of each face in the packed arrays
  double h[3], D, flin, fcub;
  const double* ia[3];     // SCALE: 1 / lambda^A of each mode per axis (mode 0: 0)
};

// Boundary value and time derivative of full-grid node (jx, jy, jz), a boundary node.
template <class T>
__device__ __forceinline__ void face_value(const BndArgs<T>& A, int jx, int jy, int jz, double& gv, double& gd) {
  const int Nx = A.nx, Ny = A.ny, Nz = A.nz;
  long long i;
  if (jx == 0 || jx == Nx) {
    i = A.off[jx == 0 ? 0 : 1] + (A.ndim == 3 ? (long long)jz * (Ny + 1) : 0LL) + jy;
  } else if (jy == 0 || jy == Ny) {
    i = A.off[jy == 0 ? 2 : 3] + (A.ndim == 3 ? (long long)jz * (Nx + 1) : 0LL) + jx;
  } else {
    i = A.off[jz == 0 ? 4 : 5] + (long long)jy * (Nx + 1) + jx;
  }
  gv = A.g[i];
  gd = A.g[A.count + i];
}

template <class T>
__global__ void __launch_bounds__(256) bnd_build_kernel(const BndArgs<T> A) {
  griddep_wait();
  const int Nx = A.nx, Ny = A.ny, Nz = A.nz;
  const bool d3 = A.ndim == 3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % Nx);
    const int y = (int)((idx / Nx) % Ny);
    const int z = (int)(idx / ((long long)Nx * Ny));
    const bool interior = x >= 1 && y >= 1 && (!d3 || z >= 1);
    const bool near = x == 1 || x == Nx - 1 || y == 1 || y == Ny - 1 || (d3 && (z == 1 || z == Nz - 1));
    double b = 0.0;
    if (interior && near) {
      const int kz = d3 ? 1 : 0;
      for (int dz = -kz; dz <= kz; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int jx = x + dx, jy = y + dy, jz = z + dz;
            const bool bnd = jx == 0 || jx == Nx || jy == 0 || jy == Ny || (d3 && (jz == 0 || jz == Nz));
            if (!bnd) continue;
            const int d[3] = {dx, dy, dz};
            double m[3], k[3];
            for (int a = 0; a < 3; ++a) {
              m[a] = A.h[a] * (d[a] == 0 ? 4.0 / 6.0 : 1.0 / 6.0);
              k[a] = (d[a] == 0 ? 2.0 : -1.0) / A.h[a];
            }
            const int na = A.ndim;
            double wm = 1.0, wk = 0.0;
            for (int a = 0; a < na; ++a) {
              wm *= m[a];
              double t = k[a];
              for (int c = 0; c < na; ++c)
                if (c != a) t *= m[c];
              wk += t;
            }
            double gv, gd;
            face_value(A, jx, jy, jz, gv, gd);
            const double fg = gv * (A.flin + A.fcub * gv * gv);
            b += wm * (fg - gd) - A.D * wk * gv;
          }
    }
    A.out[idx] = (T)b;
  }
}

template <class T>
__global__ void __launch_bounds__(256) bnd_scale_kernel(const BndArgs<T> A) {
  griddep_wait();
  const int Nx = A.nx, Ny = A.ny;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % Nx);
    const int y = (int)((idx / Nx) % Ny);
    const int z = (int)(idx / ((long long)Nx * Ny));
    double s = A.ia[0][x] * A.ia[1][y];
    if (A.ndim == 3) s *= A.ia[2][z];
    A.out[idx] = (T)((double)A.out[idx] * s);
  }
}

template <class T>
__global__ void __launch_bounds__(256) bnd_add_kernel(const BndArgs<T> A) {
  griddep_wait();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.n;
       idx += (long long)gridDim.x * blockDim.x)
    A.out[idx] += A.in[idx];
}

}  // namespace etd
