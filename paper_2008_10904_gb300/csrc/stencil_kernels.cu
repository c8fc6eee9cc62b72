// Structured-grid operators with real state: the 2-D jet advection-diffusion-
// reaction system (5-point stencil) and the 3-D three-component linearised
// advection-diffusion system (7-point stencil), and their RK4 march.
//
// Classical RK4 in low-storage form, one fused kernel per stage:
//   stage 1: k = A u   + f(t_n);        x <- u + h/2 k;  acc <- u + h/6 k;  Y <- u
//   stage 2: k = A x   + f(t_n + h/2);  x <- u + h/2 k;  acc += h/3 k
//   stage 3: k = A x   + f(t_n + h/2);  x <- u + h k;    acc += h/3 k
//   stage 4: k = A x   + f(t_n + h);    u <- acc + h/6 k
// which is algebraically the 4-stage update u + h/6 (k1 + 2k2 + 2k3 + k4).
// Stencil neighbours come through the L1/L2 caches; every stage streams
// the state-sized arrays once (coalesced along x).
//
// Adjoint operators are the exact transposes of the discrete stencils
// (discrete adjoint with identity metric): for the 2-D system the advection
// velocity U(y) is constant along x, so the transpose flips its sign; for the
// 3-D system the transposed advection uses the neighbour's velocity,
//   (A^T x)_p = (U_{p+1} x_{p+1} - U_{p-1} x_{p-1}) / (2 dx),
// and the coupling -(u . grad)U (into component x only) becomes
// -dU/dx_c * x_x into every component c.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdlib>
#include <utility>
#include <vector>

#include "rsv_ops.h"

namespace rsv {

namespace {

struct StGeom {
  int nx, ny, nz;         // nz = 1 for 2-D
  int64_t n;              // points per vector (x 3 components in 3-D)
  int kg;
  double dx, dy, dz, visc;
  const void* f0;         // ADR2D: U(y), r(y) [ny]; ADV3D: U, dU/dx, dU/dy, dU/dz [ncell]
  const void* f1;
  const void* f2;
  const void* f3;
  const void* f4;         // ADV3D, FP32: the four fields interleaved per cell (float4: U, dU/dx, dU/dy, dU/dz)
  int sponge_cells;
  double sponge_amp;
  bool adjoint;
};

template <typename R>
__device__ __forceinline__ R sponge(int i, int j, const StGeom& g) {
  int d = min(min(i, g.nx - 1 - i), min(j, g.ny - 1 - j));
  if (d >= g.sponge_cells) return R(0);
  const R s = R(g.sponge_cells);
  const R t = (s - R(d)) / s;
  return R(g.sponge_amp) * t * t;
}

// (A x) at cell (i, j) of one vector's 2-D field xv.
template <typename R>
__device__ __forceinline__ R adr2d_apply(const R* __restrict__ xv, int i, int j, const StGeom& g) {
  const R* U = reinterpret_cast<const R*>(g.f0);
  const R* rr = reinterpret_cast<const R*>(g.f1);
  const int nx = g.nx, ny = g.ny;
  const R c = xv[(int64_t)j * nx + i];
  const R w = i > 0 ? xv[(int64_t)j * nx + i - 1] : R(0);
  const R e = i < nx - 1 ? xv[(int64_t)j * nx + i + 1] : R(0);
  const R s = j > 0 ? xv[(int64_t)(j - 1) * nx + i] : R(0);
  const R nn = j < ny - 1 ? xv[(int64_t)(j + 1) * nx + i] : R(0);
  const R ux = g.adjoint ? -U[j] : U[j];
  const R idx2 = R(1) / (R(g.dx) * R(g.dx)), idy2 = R(1) / (R(g.dy) * R(g.dy)), i2dx = R(0.5) / R(g.dx);
  const R nu = R(g.visc);
  R k = (ux * i2dx + nu * idx2) * w + (-ux * i2dx + nu * idx2) * e + nu * idy2 * (s + nn);
  k += (R(-2) * nu * (idx2 + idy2) + rr[j] - sponge<R>(i, j, g)) * c;
  return k;
}

// (A x)_c for c = 0, 1, 2 at cell q of one vector (components at offsets c * ncell).
template <typename R>
__device__ __forceinline__ void adv3d_apply(const R* __restrict__ xv, int i, int j, int kz, const StGeom& g, R out[3]) {
  const R* U = reinterpret_cast<const R*>(g.f0);
  const R* Ux = reinterpret_cast<const R*>(g.f1);
  const R* Uy = reinterpret_cast<const R*>(g.f2);
  const R* Uz = reinterpret_cast<const R*>(g.f3);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t q = ((int64_t)kz * ny + j) * nx + i;
  const R idx2 = R(1) / (R(g.dx) * R(g.dx)), idy2 = R(1) / (R(g.dy) * R(g.dy)), idz2 = R(1) / (R(g.dz) * R(g.dz));
  const R i2dx = R(0.5) / R(g.dx);
  const R nu = R(g.visc);
  const R Uc = U[q];
  const R Uw = i > 0 ? U[q - 1] : R(0), Ue = i < nx - 1 ? U[q + 1] : R(0);
  R xc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R* x = xv + c * ncell;
    const R cc = x[q];
    const R w = i > 0 ? x[q - 1] : R(0);
    const R e = i < nx - 1 ? x[q + 1] : R(0);
    const R s = j > 0 ? x[q - nx] : R(0);
    const R nn = j < ny - 1 ? x[q + nx] : R(0);
    const R b = kz > 0 ? x[q - (int64_t)nx * ny] : R(0);
    const R t = kz < nz - 1 ? x[q + (int64_t)nx * ny] : R(0);
    xc[c] = cc;
    R adv;
    if (g.adjoint)
      adv = (Ue * e - Uw * w) * i2dx;
    else
      adv = -Uc * (e - w) * i2dx;
    out[c] = adv + nu * (idx2 * (w + e - R(2) * cc) + idy2 * (s + nn - R(2) * cc) + idz2 * (b + t - R(2) * cc));
  }
  if (g.adjoint) {
    out[0] -= Ux[q] * xc[0];
    out[1] -= Uy[q] * xc[0];
    out[2] -= Uz[q] * xc[0];
  } else {
    out[0] -= Ux[q] * xc[0] + Uy[q] * xc[1] + Uz[q] * xc[2];
  }
}

// Stage update at one state value given k (without forcing) and the forcing value.
template <typename R, int STAGE>
__device__ __forceinline__ void stage_update(int64_t p, R k, const R* __restrict__ u, R* __restrict__ acc,
                                             R* __restrict__ xout, R* __restrict__ ysnap, R h) {
  if (STAGE == 1) {
    const R uu = u[p];
    if (ysnap) ysnap[p] = uu;
    xout[p] = uu + R(0.5) * h * k;
    acc[p] = uu + (h / R(6)) * k;
  } else if (STAGE == 2) {
    xout[p] = u[p] + R(0.5) * h * k;
    acc[p] += (h / R(3)) * k;
  } else if (STAGE == 3) {
    xout[p] = u[p] + h * k;
    acc[p] += (h / R(3)) * k;
  } else {
    xout[p] = acc[p] + (h / R(6)) * k;  // xout is the state u here
  }
}

template <typename R, int STAGE>
__global__ void __launch_bounds__(256) adr2d_stage_kernel(StGeom g, const R* __restrict__ xin, const R* __restrict__ u,
                                                          R* __restrict__ acc, const R* __restrict__ f, R* xout,
                                                          R* __restrict__ ysnap, R h) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int v = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int64_t base = (int64_t)v * g.n;
  const int64_t p = base + (int64_t)j * g.nx + i;
  R k = adr2d_apply<R>(xin + base, i, j, g);
  if (f) k += f[p];
  stage_update<R, STAGE>(p, k, u, acc, xout, ysnap, h);
}

template <typename R, int STAGE>
__global__ void __launch_bounds__(256) adv3d_stage_kernel(StGeom g, const R* __restrict__ xin, const R* __restrict__ u,
                                                          R* __restrict__ acc, const R* __restrict__ f, R* xout,
                                                          R* __restrict__ ysnap, R h) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int jz = blockIdx.y * 8 + threadIdx.y;  // (j, kz) flattened
  const int v = blockIdx.z;
  if (i >= g.nx || jz >= g.ny * g.nz) return;
  const int j = jz % g.ny, kz = jz / g.ny;
  const int64_t base = (int64_t)v * g.n;
  const int64_t ncell = (int64_t)g.nx * g.ny * g.nz;
  R k[3];
  adv3d_apply<R>(xin + base, i, j, kz, g, k);
  const int64_t q = ((int64_t)kz * g.ny + j) * g.nx + i;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t p = base + c * ncell + q;
    R kc = k[c];
    if (f) kc += f[p];
    stage_update<R, STAGE>(p, kc, u, acc, xout, ysnap, h);
  }
}

// ---------------------------------------------------------------------------
// FP32 stage kernels, four consecutive x cells per thread (float4 loads and
// stores along x; the x neighbours of the group come from two scalar loads).
// Used when nx is a multiple of 4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float get4(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ void set4(float4& v, int q, float x) {
  if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
}

// State storage: FP32, or BF16 (RSV_PREC_BF16_STATE: storage only, arithmetic in FP32; four values
// are 8 bytes).
__device__ __forceinline__ float4 ld4s(const float* p) { return ld4(p); }
__device__ __forceinline__ float4 ld4s(const __nv_bfloat16* p) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float lds(const float* p) { return *p; }
__device__ __forceinline__ float lds(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st4s(float* p, float4 v) { st4(p, v); }
__device__ __forceinline__ void st4s(__nv_bfloat16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 o;
  o.x = *reinterpret_cast<const uint32_t*>(&a);
  o.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = o;
}

// Stage update of four values; u and the stage outputs in the state type S, accumulator, forcing
// and snapshot in FP32.
template <int STAGE, typename S>
__device__ __forceinline__ void stage_update4(int64_t p, float4 k, const S* __restrict__ u, float* __restrict__ acc,
                                              S* __restrict__ xout, float* __restrict__ ysnap, float h) {
  if (STAGE == 1) {
    const float4 uu = ld4s(u + p);
    if (ysnap) st4(ysnap + p, uu);
    st4s(xout + p, make_float4(uu.x + 0.5f * h * k.x, uu.y + 0.5f * h * k.y, uu.z + 0.5f * h * k.z, uu.w + 0.5f * h * k.w));
    const float c = h / 6.f;
    st4(acc + p, make_float4(uu.x + c * k.x, uu.y + c * k.y, uu.z + c * k.z, uu.w + c * k.w));
  } else if (STAGE == 2 || STAGE == 3) {
    const float4 uu = ld4s(u + p);
    const float cx = STAGE == 2 ? 0.5f * h : h;
    st4s(xout + p, make_float4(uu.x + cx * k.x, uu.y + cx * k.y, uu.z + cx * k.z, uu.w + cx * k.w));
    float4 a = ld4(acc + p);
    const float c = h / 3.f;
    st4(acc + p, make_float4(a.x + c * k.x, a.y + c * k.y, a.z + c * k.z, a.w + c * k.w));
  } else {
    const float4 a = ld4(acc + p);
    const float c = h / 6.f;
    st4s(xout + p, make_float4(a.x + c * k.x, a.y + c * k.y, a.z + c * k.z, a.w + c * k.w));
  }
}

template <int STAGE>
__global__ void __launch_bounds__(256) adr2d_stage4_kernel(StGeom g, const float* __restrict__ xin,
                                                           const float* __restrict__ u, float* __restrict__ acc,
                                                           const float* __restrict__ f, float* xout,
                                                           float* __restrict__ ysnap, float h) {
  const int i0 = 4 * (blockIdx.x * 32 + threadIdx.x);
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int v = blockIdx.z;
  if (i0 >= g.nx || j >= g.ny) return;
  const int nx = g.nx, ny = g.ny;
  const int64_t base = (int64_t)v * g.n;
  const float* xv = xin + base;
  const int64_t row = (int64_t)j * nx;
  const float4 c = ld4(xv + row + i0);
  const float w = i0 > 0 ? xv[row + i0 - 1] : 0.f;
  const float e = i0 + 4 < nx ? xv[row + i0 + 4] : 0.f;
  const float4 sv = j > 0 ? ld4(xv + row - nx + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 nv = j < ny - 1 ? ld4(xv + row + nx + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float* U = reinterpret_cast<const float*>(g.f0);
  const float* rr = reinterpret_cast<const float*>(g.f1);
  const float ux = g.adjoint ? -U[j] : U[j];
  const float idx2 = 1.f / ((float)g.dx * (float)g.dx), idy2 = 1.f / ((float)g.dy * (float)g.dy);
  const float i2dx = 0.5f / (float)g.dx, nu = (float)g.visc;
  const float cw = ux * i2dx + nu * idx2, ce = -ux * i2dx + nu * idx2, cy = nu * idy2;
  const float cc0 = -2.f * nu * (idx2 + idy2) + rr[j];
  float4 k;
  const float4 fv = f ? ld4(f + base + row + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float left = q == 0 ? w : get4(c, q - 1);
    const float right = q == 3 ? e : get4(c, q + 1);
    const float cc = cc0 - sponge<float>(i0 + q, j, g);
    set4(k, q, cw * left + ce * right + cy * (get4(sv, q) + get4(nv, q)) + cc * get4(c, q) + get4(fv, q));
  }
  stage_update4<STAGE, float>(base + row + i0, k, u, acc, xout, ysnap, h);
}

// Blocks are ordered with the vector index fastest, so the base-flow fields of a
// cell block are read from HBM once and served from L2 to the other vectors.
template <int STAGE, typename S>
__global__ void __launch_bounds__(256) adv3d_stage4_kernel(StGeom g, const S* __restrict__ xin,
                                                           const S* __restrict__ u, float* __restrict__ acc,
                                                           const float* __restrict__ f, S* xout,
                                                           float* __restrict__ ysnap, float h) {
  const int v = blockIdx.x % g.kg;
  const int cb = blockIdx.x / g.kg;
  const int nxb = (g.nx / 4 + 31) / 32;
  const int i0 = 4 * ((cb % nxb) * 32 + threadIdx.x);
  const int jz = (cb / nxb) * 8 + threadIdx.y;
  if (i0 >= g.nx || jz >= g.ny * g.nz) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int j = jz % ny, kz = jz / ny;
  const int64_t base = (int64_t)v * g.n;
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t q0 = ((int64_t)kz * ny + j) * nx + i0;
  const float* U = reinterpret_cast<const float*>(g.f0);
  const float* Ux = reinterpret_cast<const float*>(g.f1);
  const float* Uy = reinterpret_cast<const float*>(g.f2);
  const float* Uz = reinterpret_cast<const float*>(g.f3);
  const float idx2 = 1.f / ((float)g.dx * (float)g.dx), idy2 = 1.f / ((float)g.dy * (float)g.dy);
  const float idz2 = 1.f / ((float)g.dz * (float)g.dz), i2dx = 0.5f / (float)g.dx, nu = (float)g.visc;
  const float4 U4 = ld4(U + q0);
  const float Uw = i0 > 0 ? U[q0 - 1] : 0.f, Ue = i0 + 4 < nx ? U[q0 + 4] : 0.f;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 xc[3], k[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const S* x = xin + base + c * ncell;
    const float4 cv = ld4s(x + q0);
    const float w = i0 > 0 ? lds(x + q0 - 1) : 0.f;
    const float e = i0 + 4 < nx ? lds(x + q0 + 4) : 0.f;
    const float4 sv = j > 0 ? ld4s(x + q0 - nx) : zero;
    const float4 nv = j < ny - 1 ? ld4s(x + q0 + nx) : zero;
    const float4 bv = kz > 0 ? ld4s(x + q0 - (int64_t)nx * ny) : zero;
    const float4 tv = kz < nz - 1 ? ld4s(x + q0 + (int64_t)nx * ny) : zero;
    xc[c] = cv;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float left = q == 0 ? w : get4(cv, q - 1);
      const float right = q == 3 ? e : get4(cv, q + 1);
      const float cc = get4(cv, q);
      float adv;
      if (g.adjoint) {
        const float ul = q == 0 ? Uw : get4(U4, q - 1);
        const float ur = q == 3 ? Ue : get4(U4, q + 1);
        adv = (ur * right - ul * left) * i2dx;
      } else {
        adv = -get4(U4, q) * (right - left) * i2dx;
      }
      set4(k[c], q, adv + nu * (idx2 * (left + right - 2.f * cc) + idy2 * (get4(sv, q) + get4(nv, q) - 2.f * cc) +
                               idz2 * (get4(bv, q) + get4(tv, q) - 2.f * cc)));
    }
  }
  const float4 gx = ld4(Ux + q0), gy = ld4(Uy + q0), gz = ld4(Uz + q0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = get4(xc[0], q), x1 = get4(xc[1], q), x2 = get4(xc[2], q);
    if (g.adjoint) {
      set4(k[0], q, get4(k[0], q) - get4(gx, q) * x0);
      set4(k[1], q, get4(k[1], q) - get4(gy, q) * x0);
      set4(k[2], q, get4(k[2], q) - get4(gz, q) * x0);
    } else {
      set4(k[0], q, get4(k[0], q) - (get4(gx, q) * x0 + get4(gy, q) * x1 + get4(gz, q) * x2));
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t p = base + c * ncell + q0;
    float4 kc = k[c];
    if (f) {
      const float4 fv = ld4(f + p);
      kc = make_float4(kc.x + fv.x, kc.y + fv.y, kc.z + fv.z, kc.w + fv.w);
    }
    stage_update4<STAGE, S>(p, kc, u, acc, xout, ysnap, h);
  }
}

template <typename R>
__global__ void adr2d_apply_real_kernel(StGeom g, const R* __restrict__ x, R* __restrict__ y) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int v = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int64_t base = (int64_t)v * g.n;
  y[base + (int64_t)j * g.nx + i] = adr2d_apply<R>(x + base, i, j, g);
}

// real <-> complex helpers for the operator test entry point
template <typename R>
__global__ void split_kernel(const cpx<R>* __restrict__ x, int64_t count, R* __restrict__ re, R* __restrict__ im) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  re[e] = x[e].re;
  im[e] = x[e].im;
}
template <typename R>
__global__ void join_kernel(const R* __restrict__ re, const R* __restrict__ im, int64_t count, cpx<R>* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  y[e] = mk<R>(re[e], im[e]);
}
template <typename R>
__global__ void adv3d_apply_real_kernel(StGeom g, const R* __restrict__ x, R* __restrict__ y) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int jz = blockIdx.y * 8 + threadIdx.y;
  const int v = blockIdx.z;
  if (i >= g.nx || jz >= g.ny * g.nz) return;
  const int j = jz % g.ny, kz = jz / g.ny;
  const int64_t base = (int64_t)v * g.n;
  const int64_t ncell = (int64_t)g.nx * g.ny * g.nz;
  R k[3];
  adv3d_apply<R>(x + base, i, j, kz, g, k);
  const int64_t q = ((int64_t)kz * g.ny + j) * g.nx + i;
  for (int c = 0; c < 3; ++c) y[base + c * ncell + q] = k[c];
}

template <typename R>
rsv_status upload_real(rsv_operator op, const std::vector<double>& v, void** dst) {
  std::vector<R> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (R)v[i];
  return upload(op, o.data(), o.size() * sizeof(R), dst);
}

rsv_status upload_fields(rsv_operator op, const std::vector<std::vector<double>>& fields) {
  for (size_t a = 0; a < fields.size(); ++a) {
    rsv_status s = op->prec == RSV_PREC_FP64 ? upload_real<double>(op, fields[a], &op->fld[a])
                                             : upload_real<float>(op, fields[a], &op->fld[a]);
    if (s != RSV_OK) return s;
  }
  return RSV_OK;
}

StGeom geom_of(rsv_operator op, int kg, bool adjoint) {
  StGeom g;
  g.nx = op->nx;
  g.ny = op->ny;
  g.nz = op->kind == RSV_OP_ADV3D ? op->nz : 1;
  g.n = op->n;
  g.kg = kg;
  g.dx = op->c_dx;
  g.dy = op->c_dy;
  g.dz = op->c_dz;
  g.visc = op->visc;
  g.f0 = op->fld[0];
  g.f1 = op->fld[1];
  g.f2 = op->fld[2];
  g.f3 = op->fld[3];
  g.f4 = op->fld[4];
  g.sponge_cells = op->sponge_cells;
  g.sponge_amp = op->sponge_amp;
  g.adjoint = adjoint;
  return g;
}

// ---------------------------------------------------------------------------
// 2-D system: one whole RK4 step per launch, the four stages in shared memory.
//
// A CTA owns a TX x TY tile of one vector's field.  It reads u on the tile plus
// a 4-cell frame (one cell per stage), evaluates stage 1 on the tile plus 3
// frame cells, stage 2 on the tile plus 2, stage 3 on the tile plus 1 and
// stage 4 on the tile, so each stage's stencil finds its inputs computed by the
// previous stage in shared memory.  Cells outside the domain hold zero
// (homogeneous Dirichlet).  Per step the field is read once (the frame from
// neighbouring tiles mostly through L2), the new field written once, and the
// forcing read at the three stage times (frames included); the snapshot of u
// is written on analysed steps.  The arithmetic of each stage is that of the
// per-stage kernels above.
// ---------------------------------------------------------------------------
constexpr int kFTX = 64, kFTY = 32, kFH = 4;
constexpr int kFW = kFTX + 2 * kFH, kFHH = kFTY + 2 * kFH;
constexpr int kFThreads = 256;

template <typename R>
constexpr size_t adr2d_fused_smem() {
  // u, two stage inputs and the forcing at t_n on the frame, forcing at t_n + h/2 and
  // t_n + h, the accumulator, per-row coefficients
  return sizeof(R) * (5 * (size_t)kFW * kFHH + 2 * (size_t)kFTX * kFTY + 3 * (size_t)kFHH);
}

// Asynchronous global -> shared copy of one element (no register staging).
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(sizeof(R))
               : "memory");
}

template <typename R>
__global__ void __launch_bounds__(kFThreads) adr2d_step_kernel(StGeom g, const R* __restrict__ uin,
                                                               R* __restrict__ uout, const R* __restrict__ f0,
                                                               const R* __restrict__ fh, const R* __restrict__ f1,
                                                               R* __restrict__ ysnap, R h) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kF = kFW * kFHH;
  R* su = reinterpret_cast<R*>(smem_raw);      // u on the frame
  R* sx = su + kF;                              // stage-2 input, later stage-4 input
  R* sy = sx + kF;                              // stage-3 input
  R* sf0 = sy + kF;                             // f(t_n) on the frame
  R* sfh = sf0 + kF;                            // f(t_n + h/2) on the frame
  R* sf1 = sfh + kF;                            // f(t_n + h) on the tile
  R* sacc = sf1 + kFTX * kFTY;                  // u + h/6 k1 + h/3 k2 + h/3 k3 on the tile
  R* rw = sacc + kFTX * kFTY;                   // per frame row: west, east, centre coefficients
  R* re = rw + kFHH;
  R* rc = re + kFHH;
  const int nx = g.nx, ny = g.ny;
  const int X0 = blockIdx.x * kFTX - kFH, Y0 = blockIdx.y * kFTY - kFH;
  const int64_t base = (int64_t)blockIdx.z * g.n;
  const R idx2 = R(1) / (R(g.dx) * R(g.dx)), idy2 = R(1) / (R(g.dy) * R(g.dy));
  const R i2dx = R(0.5) / R(g.dx), nu = R(g.visc);
  const R cy = nu * idy2;
  // every input of the step is copied into shared memory up front, all copies in flight at once
  for (int e = threadIdx.x; e < kF; e += kFThreads) {
    const int li = e % kFW, lj = e / kFW;
    const int gi = X0 + li, gj = Y0 + lj;
    const bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    const int64_t p = base + (int64_t)gj * nx + gi;
    if (in) cp_async_elem(su + e, uin + p);
    else su[e] = R(0);
    const bool r1 = li >= 1 && li < kFW - 1 && lj >= 1 && lj < kFHH - 1;   // stage-1 cells
    const bool r2 = li >= 2 && li < kFW - 2 && lj >= 2 && lj < kFHH - 2;   // stage-2 and -3 cells
    if (in && r1 && f0 != nullptr) cp_async_elem(sf0 + e, f0 + p);
    else sf0[e] = R(0);
    if (in && r2 && fh != nullptr) cp_async_elem(sfh + e, fh + p);
    else sfh[e] = R(0);
  }
  for (int e = threadIdx.x; e < kFTX * kFTY; e += kFThreads) {
    const int gi = X0 + kFH + e % kFTX, gj = Y0 + kFH + e / kFTX;
    if (gi < nx && gj < ny && f1 != nullptr) cp_async_elem(sf1 + e, f1 + base + (int64_t)gj * nx + gi);
    else sf1[e] = R(0);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (threadIdx.x < kFHH) {
    const int gj = min(max(Y0 + (int)threadIdx.x, 0), ny - 1);
    const R U = reinterpret_cast<const R*>(g.f0)[gj];
    const R ux = g.adjoint ? -U : U;
    rw[threadIdx.x] = ux * i2dx + nu * idx2;
    re[threadIdx.x] = -ux * i2dx + nu * idx2;
    rc[threadIdx.x] = R(-2) * nu * (idx2 + idy2) + reinterpret_cast<const R*>(g.f1)[gj];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // k = A x at frame cell (li, lj) of the shared field x, plus the forcing value
  auto apply = [&](const R* x, int li, int lj, int gi, int gj, R fv) -> R {
    const int e = lj * kFW + li;
    const R cc = rc[lj] - sponge<R>(gi, gj, g);
    return rw[lj] * x[e - 1] + re[lj] * x[e + 1] + cy * (x[e - kFW] + x[e + kFW]) + cc * x[e] + fv;
  };
#pragma unroll 1
  for (int stage = 1; stage <= 3; ++stage) {
    const int m = stage;                              // frame cells skipped on each side
    const int w = kFW - 2 * m, hh = kFHH - 2 * m;
    const R* xin = stage == 1 ? su : stage == 2 ? sx : sy;
    R* xout = stage == 1 ? sx : stage == 2 ? sy : sx;
    const R* sf = stage == 1 ? sf0 : sfh;
    const R cx = stage == 3 ? h : R(0.5) * h;
    const R ca = stage == 1 ? h / R(6) : h / R(3);
    for (int e = threadIdx.x; e < w * hh; e += kFThreads) {
      const int li = m + e % w, lj = m + e / w;
      const int gi = X0 + li, gj = Y0 + lj;
      const int le = lj * kFW + li;
      R xo = R(0);
      if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
        const R k = apply(xin, li, lj, gi, gj, sf[le]);
        const R uu = su[le];
        xo = uu + cx * k;
        const int ti = li - kFH, tj = lj - kFH;
        if (ti >= 0 && ti < kFTX && tj >= 0 && tj < kFTY) {
          if (stage == 1) {
            sacc[tj * kFTX + ti] = uu + ca * k;
            if (ysnap != nullptr) ysnap[base + (int64_t)gj * nx + gi] = uu;
          } else {
            sacc[tj * kFTX + ti] += ca * k;
          }
        }
      }
      // stage 3 writes into the stage-2 input: the barrier after stage 2 separates them
      xout[le] = xo;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kFTX * kFTY; e += kFThreads) {
    const int ti = e % kFTX, tj = e / kFTX;
    const int li = kFH + ti, lj = kFH + tj;
    const int gi = X0 + li, gj = Y0 + lj;
    if (gi < nx && gj < ny) {
      const R k = apply(sx, li, lj, gi, gj, sf1[e]);
      uout[base + (int64_t)gj * nx + gi] = sacc[e] + (h / R(6)) * k;
    }
  }
}

template <typename R>
cudaError_t launch_adr2d_step(rsv_operator op, const StGeom& g, const R* uin, R* uout, const R* f0, const R* fh,
                              const R* f1, R* ysnap, R h) {
  // per-device attribute: set before every launch (cheap next to a step over the whole grid)
  cudaError_t ae = cudaFuncSetAttribute(adr2d_step_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)adr2d_fused_smem<R>());
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)((g.nx + kFTX - 1) / kFTX), (unsigned)((g.ny + kFTY - 1) / kFTY), (unsigned)g.kg);
  adr2d_step_kernel<R><<<grid, kFThreads, adr2d_fused_smem<R>(), op->stream>>>(g, uin, uout, f0, fh, f1, ysnap, h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 3-D system, FP32: RK4 in two launches per step, each fusing a pair of stages.
//
//   pair A (stages 1, 2):  k1 = A u + f(t_n)        on the tile + 1 halo cell in x, y
//                          x2 = u + h/2 k1           (shared memory)
//                          k2 = A x2 + f(t_n + h/2)  on the tile
//                          x3 = u + h/2 k2,  acc = u + h/6 k1 + h/3 k2,  Y <- u
//   pair B (stages 3, 4):  k3 = A x3 + f(t_n + h/2)  on the tile + 1 halo cell in x, y
//                          x4 = u + h k3             (shared memory)
//                          k4 = A x4 + f(t_n + h)    on the tile
//                          u' = acc + h/3 k3 + h/6 k4
// which is the classical RK4 update u + h/6 (k1 + 2 k2 + 2 k3 + k4).  h/6 k1 and h/3 k3
// are recovered from the stage values in shared memory, (x2 - u)/3 and (x4 - u)/3.
//
// A CTA owns a TX x TY tile in (x, y) of one vector and a run of ZC planes in z, and
// streams through z: the stencil input of the first stage of the pair (u or x3) sits in a
// ring of four planes with two halo cells in x and y (three planes in use, the next one
// arriving by asynchronous copies), the intermediate stage (x2 or x4) in a ring of three
// planes with one halo cell.  At plane p the first stage is evaluated on plane p + 1 and
// the second on plane p, one barrier apart.  Per step the state-sized arrays cross HBM
// about 11 times (pair A: u, two forcing samples read, x3 and acc written, plus the
// snapshot on analysed steps; pair B: x3, u, acc and two forcing samples read, u' written)
// against about 20 for the four single-stage kernels; halo cells come from L2.
// Cells outside the grid hold zero (homogeneous Dirichlet), in both rings.
// ---------------------------------------------------------------------------
// Tile width and the ring row widths; each kernel variant derives its heights from its tile height.
constexpr int k3TX = 64, k3ZC = 16;
constexpr int k3UW = k3TX + 8;     // ring of the pair's stencil input: x from X0 - 4 (16-byte aligned
                                   // rows), halo 2 used; y halo 2
constexpr int k3XW = k3TX + 2;     // ring of the intermediate stage (halo 1)
constexpr int k3Row4 = k3UW / 4;   // 16-byte chunks per ring row (18)

struct Pair3D {
  const float* in;     // stencil input of the first stage: u (pair A) or x3 (pair B)
  const float* u;      // pair B: the state u (pair A reads u as `in`)
  const float* acc;    // pair B: accumulator from pair A
  const float* fa;     // forcing of the first stage: f(t_n) (A) or f(t_n + h/2) (B); nullable
  const float* fb;     // forcing of the second stage: f(t_n + h/2) (A) or f(t_n + h) (B); nullable
  float* out;          // pair A: x3; pair B: u'
  float* acc_out;      // pair A: accumulator
  float* ysnap;        // pair A: snapshot of u (nullable)
  float h;
  int zchunks;         // z is cut into this many runs of planes, as even as possible
};

// Base flow at one cell, as the operator's fields hold it (U = erf(r / delta(x)) and its gradient):
// forward advection uses U at the cell, the transposed advection U at the two x neighbours.
struct Bf {
  float Uc, Uw, Ue, Ux, Uy, Uz;
};

// 7-point operator (forward or transposed) of component-interleaved shared-memory planes at index e
// of a plane with rows of width W; planes below, centre, above.
template <bool ADJ, int W, int PLANE>
__device__ __forceinline__ void op3d_smem(const float* __restrict__ xb, const float* __restrict__ xc,
                                          const float* __restrict__ xt, int e, const Bf& bf, float cdx,
                                          float idx2, float idy2, float idz2, float nu, float out[3]) {
  float xcen[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* pc = xc + c * PLANE;
    const float cc = pc[e], w = pc[e - 1], ee = pc[e + 1], s = pc[e - W], n = pc[e + W];
    const float b = xb[c * PLANE + e], t = xt[c * PLANE + e];
    xcen[c] = cc;
    const float adv = ADJ ? (bf.Ue * ee - bf.Uw * w) * cdx : -bf.Uc * (ee - w) * cdx;
    out[c] = adv + nu * (idx2 * (w + ee - 2.f * cc) + idy2 * (s + n - 2.f * cc) + idz2 * (b + t - 2.f * cc));
  }
  if (ADJ) {
    out[0] -= bf.Ux * xcen[0];
    out[1] -= bf.Uy * xcen[0];
    out[2] -= bf.Uz * xcen[0];
  } else {
    out[0] -= bf.Ux * xcen[0] + bf.Uy * xcen[1] + bf.Uz * xcen[2];
  }
}

// Base-flow fields at cell offset q (x index i), for the forward or transposed operator.
// Forward: one 16-byte load of the interleaved fields.  Transposed: U at the two x neighbours and
// the gradient as separate loads (the interleaved load measured 12% slower there).
template <bool ADJ>
__device__ __forceinline__ Bf load_bf(const StGeom& g, int q, int i, bool ok) {
  const float* U = reinterpret_cast<const float*>(g.f0);
  Bf b;
  if (!ADJ) {
    const float4 v = ok ? __ldg(reinterpret_cast<const float4*>(g.f4) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    b.Uc = v.x;
    b.Uw = b.Ue = 0.f;
    b.Ux = v.y;
    b.Uy = v.z;
    b.Uz = v.w;
    return b;
  }
  const float* Ux = reinterpret_cast<const float*>(g.f1);
  const float* Uy = reinterpret_cast<const float*>(g.f2);
  const float* Uz = reinterpret_cast<const float*>(g.f3);
  b.Uc = 0.f;
  b.Uw = (ok && i > 0) ? __ldg(U + q - 1) : 0.f;
  b.Ue = (ok && i < g.nx - 1) ? __ldg(U + q + 1) : 0.f;
  b.Ux = ok ? __ldg(Ux + q) : 0.f;
  b.Uy = ok ? __ldg(Uy + q) : 0.f;
  b.Uz = ok ? __ldg(Uz + q) : 0.f;
  return b;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// Per-thread registers of one plane's point inputs, loaded one plane ahead of their use.
template <int S1>
struct Stage1In {
  float f[S1][3];      // forcing of the first stage
  float u[S1][3];      // pair B: the state u
  Bf bf[S1];           // base flow
};
template <int S2>
struct Stage2In {
  float f[S2][3];      // forcing of the second stage
  float u[S2][3];      // pair B: the state u
  float a[S2][3];      // pair B: the accumulator
  Bf bf[S2];           // base flow
};

// Tile height TY and threads NT of a pair-kernel variant: 64 x 8 with 256 threads (two CTAs per SM)
// or 64 x 16 with 512 threads (one CTA per SM, less halo work per output cell).
template <int TY>
constexpr size_t pair3d_smem() {
  return sizeof(float) * (4 * 3 * (size_t)((k3TX + 8) * (TY + 4)) + 3 * 3 * (size_t)((k3TX + 2) * (TY + 2)));
}

// Requires nx % 4 == 0 (16-byte rows of the input ring) and n < 2^31 (32-bit offsets in a vector).
template <bool ADJ, bool PAIR_B, int MINB, int TY, int NT>
__global__ void __launch_bounds__(NT, MINB) adv3d_pair_kernel(StGeom g, Pair3D P) {
  // this variant's tile geometry (heights and slots follow from its tile height TY and threads NT)
  constexpr int k3TY = TY, k3Threads = NT;
  constexpr int k3UH = k3TY + 4, k3XH = k3TY + 2;
  constexpr int k3UP = k3UW * k3UH, k3XP = k3XW * k3XH;
  constexpr int k3S1 = (k3XP + k3Threads - 1) / k3Threads;
  constexpr int k3S2 = k3TX * k3TY / k3Threads;
  static_assert(k3TX * k3TY % k3Threads == 0, "whole second-stage cells per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);            // [4 planes][3 comps][k3UP]
  float* mid = ring + 4 * 3 * k3UP;                              // [3 planes][3 comps][k3XP]
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ncell = nx * ny * nz;
  const int plane = nx * ny;
  // block order: vector fastest (neighbouring tiles of all vectors in flight together), then x, y, z
  int b = blockIdx.x;
  const int v = b % g.kg;
  b /= g.kg;
  const int ntx = (nx + k3TX - 1) / k3TX, nty = (ny + k3TY - 1) / k3TY;
  const int X0 = (b % ntx) * k3TX;
  b /= ntx;
  const int Y0 = (b % nty) * k3TY;
  const int cz = b / nty;
  const int z0 = (int)((int64_t)cz * nz / P.zchunks);
  const int z1 = (int)((int64_t)(cz + 1) * nz / P.zchunks);
  const int64_t base = (int64_t)v * g.n;
  const float* __restrict__ in = P.in + base;
  const float* __restrict__ fa = P.fa ? P.fa + base : nullptr;
  const float* __restrict__ fb = P.fb ? P.fb + base : nullptr;
  const float* __restrict__ pu = PAIR_B ? P.u + base : nullptr;
  const float* __restrict__ pacc = PAIR_B ? P.acc + base : nullptr;
  float* __restrict__ out = P.out + base;
  float* __restrict__ acc_out = PAIR_B ? nullptr : P.acc_out + base;
  float* __restrict__ ysnap = P.ysnap ? P.ysnap + base : nullptr;
  const float cdx = 0.5f / (float)g.dx, idx2 = 1.f / ((float)g.dx * (float)g.dx);
  const float idy2 = 1.f / ((float)g.dy * (float)g.dy), idz2 = 1.f / ((float)g.dz * (float)g.dz);
  const float nu = (float)g.visc;
  const float h = P.h;
  const float c1 = PAIR_B ? h : 0.5f * h;       // x_mid = u + c1 (A x + f_a)
  const float c2 = PAIR_B ? h / 6.f : 0.5f * h;  // pair A: x3 = u + h/2 k2; pair B: u' = ... + h/6 k4
  const int tid = threadIdx.x;
  // Launched as a programmatic dependent of the previous pair kernel, the CTA may be resident before
  // that kernel ends: it waits for it here, before any memory access (a no-op after an ordinary
  // launch), and then lets the next kernel launch, whose CTAs wait in the same place.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // The forward first stage evaluates all its slots as one straight-line block (masked afterwards);
  // the transposed one (five base-flow values per cell) keeps a branch per slot, which holds it
  // under the register limit without spills (the flat form spilled and measured 2.3% slower).
  constexpr bool kFlat1 = !ADJ;

  // per-thread cells, fixed over the planes: (x, y) offset in a plane (-1 outside the grid), x index,
  // and the shared-memory indices in the input ring and the intermediate ring
  int xy1[k3S1], gi1[k3S1], eu1[k3S1];
#pragma unroll
  for (int sl = 0; sl < k3S1; ++sl) {
    const int e = tid + sl * k3Threads;
    const int lx = e % k3XW, ly = e / k3XW;
    const int gi = X0 - 1 + lx, gj = Y0 - 1 + ly;
    const bool ok = e < k3XP && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    xy1[sl] = ok ? gj * nx + gi : -1;
    gi1[sl] = gi;
    // ring x index = gi - (X0 - 4); a slot past the region evaluates (and discards) the first cell
    eu1[sl] = e < k3XP ? (ly + 1) * k3UW + lx + 3 : k3UW + 3;
  }
  int xy2[k3S2], gi2[k3S2];
#pragma unroll
  for (int sl = 0; sl < k3S2; ++sl) {
    const int e = tid + sl * k3Threads;
    const int gi = X0 + e % k3TX, gj = Y0 + e / k3TX;
    xy2[sl] = (gi < nx && gj < ny) ? gj * nx + gi : -1;
    gi2[sl] = gi;
  }

  // asynchronous copy of plane kz of the stencil input into ring slot kz & 3: rows of 72 floats from
  // x = X0 - 4, 16-byte chunks, each wholly inside or outside the grid (nx and X0 are multiples of 4)
  auto load_plane = [&](int kz) {
    float* dst = ring + (size_t)(kz & 3) * 3 * k3UP;
    const bool zin = kz >= 0 && kz < nz;
    for (int e = tid; e < 3 * k3UH * k3Row4; e += k3Threads) {
      const int row = e / k3Row4, ch = e - row * k3Row4;      // row = c * k3UH + ly
      const int c = row / k3UH, ly = row - c * k3UH;
      const int gj = Y0 - 2 + ly, gx = X0 - 4 + 4 * ch;
      float* d = dst + c * k3UP + ly * k3UW + 4 * ch;
      if (zin && gj >= 0 && gj < ny && gx >= 0 && gx < nx)
        cp_async16(d, in + c * ncell + kz * plane + gj * nx + gx);
      else
        *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto fetch1 = [&](int kz, Stage1In<k3S1>& r) {
    const bool zin = kz >= 0 && kz < nz;
#pragma unroll
    for (int sl = 0; sl < k3S1; ++sl) {
      const bool ok = zin && xy1[sl] >= 0;
      const int q = kz * plane + xy1[sl];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r.f[sl][c] = (ok && fa) ? __ldg(fa + q + c * ncell) : 0.f;
        r.u[sl][c] = (PAIR_B && ok) ? __ldg(pu + q + c * ncell) : 0.f;
      }
      r.bf[sl] = load_bf<ADJ>(g, q, gi1[sl], ok);
    }
  };
  auto fetch2 = [&](int kz, Stage2In<k3S2>& r) {
    const bool zin = kz >= z0 && kz < z1;
#pragma unroll
    for (int sl = 0; sl < k3S2; ++sl) {
      const bool ok = zin && xy2[sl] >= 0;
      const int q = kz * plane + xy2[sl];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r.f[sl][c] = (ok && fb) ? __ldg(fb + q + c * ncell) : 0.f;
        r.u[sl][c] = (PAIR_B && ok) ? __ldg(pu + q + c * ncell) : 0.f;
        r.a[sl][c] = (PAIR_B && ok) ? __ldg(pacc + q + c * ncell) : 0.f;
      }
      r.bf[sl] = load_bf<ADJ>(g, q, gi2[sl], ok);
    }
  };

  // first stage on plane kz, tile + 1 halo cell: x_mid = u + c1 (A x + f_a); zero outside the grid.
  // In the flat form every slot is evaluated (cells outside the grid read zeros) and masked
  // afterwards, so the slots form one straight-line block whose loads and arithmetic the compiler
  // can interleave.
  auto first_stage = [&](int kz, const Stage1In<k3S1>& r) {
    float* dst = mid + (size_t)(((kz % 3) + 3) % 3) * 3 * k3XP;
    const float* xb = ring + (size_t)((kz - 1) & 3) * 3 * k3UP;
    const float* xc = ring + (size_t)(kz & 3) * 3 * k3UP;
    const float* xt = ring + (size_t)((kz + 1) & 3) * 3 * k3UP;
    const bool zin = kz >= 0 && kz < nz;
#pragma unroll
    for (int sl = 0; sl < k3S1; ++sl) {
      const int e = tid + sl * k3Threads;
      if (!kFlat1 && e >= k3XP) break;
      const bool ok = zin && xy1[sl] >= 0;
      float xo[3] = {0.f, 0.f, 0.f};
      if (kFlat1 || ok) {
        float k[3];
        op3d_smem<ADJ, k3UW, k3UP>(xb, xc, xt, eu1[sl], r.bf[sl], cdx, idx2, idy2, idz2, nu, k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float uu = PAIR_B ? r.u[sl][c] : xc[c * k3UP + eu1[sl]];
          xo[c] = ok ? uu + c1 * (k[c] + r.f[sl][c]) : 0.f;
        }
      }
      if (e < k3XP) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[c * k3XP + e] = xo[c];
      }
    }
  };

  // second stage on plane kz, the tile
  auto second_stage = [&](int kz, const Stage2In<k3S2>& r) {
    const float* mb = mid + (size_t)((((kz - 1) % 3) + 3) % 3) * 3 * k3XP;
    const float* mc = mid + (size_t)(kz % 3) * 3 * k3XP;
    const float* mt = mid + (size_t)((kz + 1) % 3) * 3 * k3XP;
    const float* uc = ring + (size_t)(kz & 3) * 3 * k3UP;
    // every slot is evaluated (its indices are inside the tile) and only the stores are masked
#pragma unroll
    for (int sl = 0; sl < k3S2; ++sl) {
      const int e = tid + sl * k3Threads;
      const int tx = e % k3TX, ty = e / k3TX;
      const int em = (ty + 1) * k3XW + tx + 1;
      const int q = kz * plane + xy2[sl];
      float k[3];
      op3d_smem<ADJ, k3XW, k3XP>(mb, mc, mt, em, r.bf[sl], cdx, idx2, idy2, idz2, nu, k);
      if (xy2[sl] < 0) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int pidx = c * ncell + q;
        const float xm = mc[c * k3XP + em];
        if (!PAIR_B) {
          const float uu = uc[c * k3UP + (ty + 2) * k3UW + tx + 4];
          const float kk = k[c] + r.f[sl][c];
          out[pidx] = uu + c2 * kk;                                       // x3
          acc_out[pidx] = uu + (xm - uu) * (1.f / 3.f) + (h / 3.f) * kk;   // u + h/6 k1 + h/3 k2
          if (ysnap) ysnap[pidx] = uu;
        } else {
          const float uu = r.u[sl][c];
          const float a = r.a[sl][c] + (xm - uu) * (1.f / 3.f);           // + h/3 k3
          out[pidx] = a + c2 * (k[c] + r.f[sl][c]);                       // + h/6 k4
        }
      }
    }
  };

  Stage1In<k3S1> s1;
  Stage2In<k3S2> s2;
  // prologue: planes z0 - 2 .. z0 + 1 of the stencil input; first stage on plane z0 - 1
  for (int kz = z0 - 2; kz <= z0 + 1; ++kz) load_plane(kz);
  fetch1(z0 - 1, s1);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  first_stage(z0 - 1, s1);
  fetch1(z0, s1);
  fetch2(z0, s2);
  for (int p = z0 - 1; p < z1; ++p) {
    // plane p + 2 has landed; the slot of plane p - 1 is free and receives plane p + 3
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (p + 3 <= z1 + 1) load_plane(p + 3);
    first_stage(p + 1, s1);
    if (p + 2 <= z1) fetch1(p + 2, s1);         // in flight during the barrier and the second stage
    __syncthreads();
    if (p >= z0) {
      second_stage(p, s2);
      if (p + 1 < z1) fetch2(p + 1, s2);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// 2-D system, FP32: RK4 in two launches per step, each fusing a pair of stages (the scheme of the
// 3-D pair kernels above, on one plane).  A CTA owns a 64 x 32 tile of one vector: the pair's
// stencil input (u or x3) is copied with a halo of two cells into shared memory (16-byte
// asynchronous copies of rows from x = X0 - 4), the first stage is evaluated on the tile and a
// one-cell halo into a second shared array, the second stage on the tile.  Per step the
// state-sized arrays cross HBM about 11 times (pair A: u and two forcing samples read, x3 and acc
// written, plus the snapshot on analysed steps; pair B: x3, u, acc and two forcing samples read,
// u' written) against about 20 for the four single-stage kernels.  Cells outside the grid hold zero.
// ---------------------------------------------------------------------------
constexpr int k2TX = 64, k2TY = 32, k2Threads = 256;
constexpr int k2UW = k2TX + 8, k2UH = k2TY + 4;     // input tile: x from X0 - 4, y halo 2
constexpr int k2XW = k2TX + 2, k2XH = k2TY + 2;     // first-stage tile: halo 1

// Sponge rate at cell (gi, gj) with precomputed 1 / sponge_cells (the same values as sponge()).
__device__ __forceinline__ float sponge_fast(int gi, int gj, const StGeom& g, float inv_s) {
  const int d = min(min(gi, g.nx - 1 - gi), min(gj, g.ny - 1 - gj));
  if (d >= g.sponge_cells) return 0.f;
  const float t = (float)(g.sponge_cells - d) * inv_s;
  return (float)g.sponge_amp * t * t;
}

// Shared-memory tiles of the 2-D pair kernel (floats): the stencil input (rows Y0-2 .. Y0+33, x from
// X0-4, 72 wide), the first stage's forcing and (pair B) state on its halo region (rows Y0-1 ..
// Y0+32, 72 wide), the first-stage result (66 x 34), and the second stage's forcing and (pair B)
// accumulator on the tile (64 x 32).  Every global read of the kernel is one of these 16-byte
// asynchronous copies, issued together at the start.
constexpr int k2HW = k2UW, k2HH = k2XH;            // halo-region tiles: 72 x 34
constexpr int k2Smem = (k2UH * k2UW + 2 * k2HH * k2HW + k2XH * k2XW + 2 * k2TX * k2TY) * 4;

// Copies rows [y0, y0 + nrow) x [x0, x0 + 4 nch) of a field into a tile with rows of width w (16-byte
// chunks, wholly inside the grid or zero).
__device__ __forceinline__ void tile_copy(float* t, int w, const float* src, int x0, int nch, int y0, int nrow,
                                          int nx, int ny, int tid) {
  for (int e = tid; e < nrow * nch; e += k2Threads) {
    const int ly = e / nch, ch = e - ly * nch;
    const int gj = y0 + ly, gx = x0 + 4 * ch;
    float* d = t + ly * w + 4 * ch;
    if (src != nullptr && gj >= 0 && gj < ny && gx >= 0 && gx < nx)
      cp_async16(d, src + (int64_t)gj * nx + gx);
    else
      *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Requires nx % 4 == 0 (16-byte rows of the tiles and of the second stage's float4 stores).
template <bool PAIR_B>
__global__ void __launch_bounds__(k2Threads) adr2d_pair_kernel(StGeom g, Pair3D P) {
  extern __shared__ __align__(16) unsigned char smem2[];
  float* tin = reinterpret_cast<float*>(smem2);        // [k2UH][k2UW]
  float* ta = tin + k2UH * k2UW;                        // [k2HH][k2HW] forcing of the first stage
  float* tu = ta + k2HH * k2HW;                         // [k2HH][k2HW] pair B: the state u
  float* mid = tu + k2HH * k2HW;                        // [k2XH][k2XW]
  float* tb = mid + k2XH * k2XW;                        // [k2TY][k2TX] forcing of the second stage
  float* tc = tb + k2TX * k2TY;                         // [k2TY][k2TX] pair B: the accumulator
  __shared__ float rowc[k2XH][3];            // per row of the first-stage tile: cw, ce, diagonal without sponge
  const int nx = g.nx, ny = g.ny;
  int b = blockIdx.x;
  const int v = b % g.kg;       // vector fastest: the tiles of all vectors of a region run together
  b /= g.kg;
  const int ntx = (nx + k2TX - 1) / k2TX;
  const int X0 = (b % ntx) * k2TX, Y0 = (b / ntx) * k2TY;
  const int64_t base = (int64_t)v * g.n;
  float* __restrict__ out = P.out + base;
  float* __restrict__ acc_out = PAIR_B ? nullptr : P.acc_out + base;
  float* __restrict__ ysnap = P.ysnap ? P.ysnap + base : nullptr;
  const float i2dx = 0.5f / (float)g.dx, idx2 = 1.f / ((float)g.dx * (float)g.dx);
  const float idy2 = 1.f / ((float)g.dy * (float)g.dy), nu = (float)g.visc;
  const float cy = nu * idy2;
  const float inv_s = g.sponge_cells > 0 ? 1.f / (float)g.sponge_cells : 0.f;
  // the sponge touches this tile (with its halo) only near a wall
  const bool near_wall = X0 - 1 < g.sponge_cells || X0 + k2TX + 1 > nx - g.sponge_cells || Y0 - 1 < g.sponge_cells ||
                         Y0 + k2TY + 1 > ny - g.sponge_cells;
  const float h = P.h;
  const float c1 = PAIR_B ? h : 0.5f * h;
  const float c2 = PAIR_B ? h / 6.f : 0.5f * h;
  const int tid = threadIdx.x;
  tile_copy(tin, k2UW, P.in + base, X0 - 4, k2UW / 4, Y0 - 2, k2UH, nx, ny, tid);
  tile_copy(ta, k2HW, P.fa ? P.fa + base : nullptr, X0 - 4, k2HW / 4, Y0 - 1, k2HH, nx, ny, tid);
  if (PAIR_B) tile_copy(tu, k2HW, P.u + base, X0 - 4, k2HW / 4, Y0 - 1, k2HH, nx, ny, tid);
  tile_copy(tb, k2TX, P.fb ? P.fb + base : nullptr, X0, k2TX / 4, Y0, k2TY, nx, ny, tid);
  if (PAIR_B) tile_copy(tc, k2TX, P.acc + base, X0, k2TX / 4, Y0, k2TY, nx, ny, tid);
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (tid < k2XH) {   // row coefficients of rows Y0 - 1 .. Y0 + k2TY
    const int gj = min(max(Y0 - 1 + tid, 0), ny - 1);
    const float* U = reinterpret_cast<const float*>(g.f0);
    const float* rr = reinterpret_cast<const float*>(g.f1);
    const float ux = g.adjoint ? -__ldg(U + gj) : __ldg(U + gj);
    rowc[tid][0] = ux * i2dx + nu * idx2;
    rowc[tid][1] = -ux * i2dx + nu * idx2;
    rowc[tid][2] = -2.f * nu * (idx2 + idy2) + __ldg(rr + gj);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // first stage on the tile and a one-cell halo: x_mid = u + c1 (A x + f_a); zero outside the grid
  for (int e = tid; e < k2XH * k2XW; e += k2Threads) {
    const int lx = e % k2XW, ly = e / k2XW;
    const int gi = X0 - 1 + lx, gj = Y0 - 1 + ly;
    float xo = 0.f;
    if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
      const int et = (ly + 1) * k2UW + lx + 3;      // tin index of (gi, gj)
      const int eh = ly * k2HW + lx + 3;            // halo-region tile index of (gi, gj)
      const float cc = rowc[ly][2] - (near_wall ? sponge_fast(gi, gj, g, inv_s) : 0.f);
      const float k = rowc[ly][0] * tin[et - 1] + rowc[ly][1] * tin[et + 1] + cy * (tin[et - k2UW] + tin[et + k2UW]) +
                      cc * tin[et] + ta[eh];
      const float uu = PAIR_B ? tu[eh] : tin[et];
      xo = uu + c1 * k;
    }
    mid[e] = xo;
  }
  __syncthreads();
  // second stage on the tile, four cells along x per item (16-byte stores)
  for (int e = tid; e < k2TX * k2TY / 4; e += k2Threads) {
    const int tx = 4 * (e % (k2TX / 4)), ty = e / (k2TX / 4);
    const int gi0 = X0 + tx, gj = Y0 + ty;
    if (gi0 >= nx || gj >= ny) continue;
    const int64_t q = (int64_t)gj * nx + gi0;
    const int ly = ty + 1;                          // row of the first-stage tile
    const float cw = rowc[ly][0], ce = rowc[ly][1], cd = rowc[ly][2];
    float4 kk, xm;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int em = ly * k2XW + tx + c + 1;
      const float cc = cd - (near_wall ? sponge_fast(gi0 + c, gj, g, inv_s) : 0.f);
      const float k = cw * mid[em - 1] + ce * mid[em + 1] + cy * (mid[em - k2XW] + mid[em + k2XW]) + cc * mid[em] +
                      tb[ty * k2TX + tx + c];
      set4(kk, c, k);
      set4(xm, c, mid[em]);
    }
    if (!PAIR_B) {
      const float* urow = tin + (ty + 2) * k2UW + tx + 4;
      const float4 uu = make_float4(urow[0], urow[1], urow[2], urow[3]);
      float4 o3, oa;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float u1 = get4(uu, c), k = get4(kk, c);
        set4(o3, c, u1 + c2 * k);                                             // x3
        set4(oa, c, u1 + (get4(xm, c) - u1) * (1.f / 3.f) + (h / 3.f) * k);  // u + h/6 k1 + h/3 k2
      }
      st4(out + q, o3);
      st4(acc_out + q, oa);
      if (ysnap) st4(ysnap + q, uu);
    } else {
      const float* urow = tu + (ty + 1) * k2HW + tx + 4;
      float4 o;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float u1 = urow[c];
        const float a = tc[ty * k2TX + tx + c] + (get4(xm, c) - u1) * (1.f / 3.f);   // + h/3 k3
        set4(o, c, a + c2 * get4(kk, c));                                           // + h/6 k4
      }
      st4(out + q, o);
    }
  }
}

template <bool PAIR_B>
cudaError_t launch_pair2d(rsv_operator op, const StGeom& g, const Pair3D& P) {
  // per-device attribute: set before every launch (cheap next to a pass over the field)
  cudaError_t e = cudaFuncSetAttribute(adr2d_pair_kernel<PAIR_B>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2Smem);
  if (e != cudaSuccess) return e;
  const unsigned ntx = (unsigned)((g.nx + k2TX - 1) / k2TX), nty = (unsigned)((g.ny + k2TY - 1) / k2TY);
  adr2d_pair_kernel<PAIR_B><<<ntx * nty * (unsigned)g.kg, k2Threads, k2Smem, op->stream>>>(g, P);
  return cudaGetLastError();
}

// Resident CTAs per SM the pair kernels are compiled for: 2 (no spills, the default) or 3 (80
// registers, spills); RSV_PAIR3D_MINB selects (read once per process).
int pair3d_minb() {
  static int v = [] {
    const char* e = getenv("RSV_PAIR3D_MINB");
    return (e != nullptr && e[0] == '3') ? 3 : 2;
  }();
  return v;
}

// Number of z runs: as many CTAs as fill whole waves of the resident CTAs (runs of at least 4 planes,
// at most 64 of them), so that the last wave is not left mostly idle.
int pair3d_zchunks(int per_chunk, int nz, int resident) {
  int best = std::max(1, (nz + k3ZC - 1) / k3ZC);
  double best_eff = -1.0;
  for (int nc = std::max(1, nz / 64); nc <= std::min(64, std::max(1, nz / 4)); ++nc) {
    const double waves = (double)per_chunk * nc / std::max(resident, 1);
    const double eff = waves / std::ceil(waves) - 0.002 * nc;     // prefer fewer runs (less halo work)
    if (eff > best_eff) {
      best_eff = eff;
      best = nc;
    }
  }
  return best;
}

// Programmatic dependent launch of the pair kernels: on (default) or off (RSV_PAIR3D_PDL=0), read once
// per process.
bool pair3d_pdl() {
  static bool v = [] {
    const char* e = getenv("RSV_PAIR3D_PDL");
    return !(e != nullptr && e[0] == '0');
  }();
  return v;
}

template <bool ADJ, bool PAIR_B, int MINB, int TY, int NT>
cudaError_t launch_pair3d_minb(rsv_operator op, const StGeom& g, const Pair3D& P0) {
  constexpr size_t smem = pair3d_smem<TY>();
  // the shared-memory opt-in and the residency are per device; set up once per device under a lock
  static std::mutex mu;
  static int resident_dev[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int resident = std::max(1, op->sm_count);
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || resident_dev[dev] == 0) {
      cudaError_t e = cudaFuncSetAttribute(adv3d_pair_kernel<ADJ, PAIR_B, MINB, TY, NT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adv3d_pair_kernel<ADJ, PAIR_B, MINB, TY, NT>, NT,
                                                        smem);
      if (e != cudaSuccess) return e;
      resident = std::max(1, per_sm) * std::max(1, op->sm_count);
      if (dev >= 0 && dev < 64) resident_dev[dev] = resident;
    } else {
      resident = resident_dev[dev];
    }
  }
  const unsigned ntx = (unsigned)((g.nx + k3TX - 1) / k3TX), nty = (unsigned)((g.ny + TY - 1) / TY);
  Pair3D P = P0;
  P.zchunks = pair3d_zchunks((int)(ntx * nty) * g.kg, g.nz, resident);
  const unsigned blocks = ntx * nty * (unsigned)P.zchunks * (unsigned)g.kg;
  // programmatic dependent launch: the kernel may start as the previous one drains (the kernel
  // orders its reads and writes around griddepcontrol.wait)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = op->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pair3d_pdl() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, adv3d_pair_kernel<ADJ, PAIR_B, MINB, TY, NT>, g, P);
}

// Tile height of the pair kernels: 8 (default) or 16 (RSV_PAIR3D_TY=16), read once per process.
int pair3d_ty() {
  static int v = [] {
    const char* e = getenv("RSV_PAIR3D_TY");
    return (e != nullptr && atoi(e) == 16) ? 16 : 8;
  }();
  return v;
}

template <bool ADJ, bool PAIR_B>
cudaError_t launch_pair3d(rsv_operator op, const StGeom& g, const Pair3D& P) {
  if (pair3d_ty() == 16) return launch_pair3d_minb<ADJ, PAIR_B, 1, 16, 512>(op, g, P);
  return pair3d_minb() == 2 ? launch_pair3d_minb<ADJ, PAIR_B, 2, 8, 256>(op, g, P)
                            : launch_pair3d_minb<ADJ, PAIR_B, 3, 8, 256>(op, g, P);
}

// RSV_STENCIL_FUSED=1 selects the whole-step kernel (read at each march tile).  The
// per-stage float4 kernels stay the default: on GB300 they measured 5% faster at the
// 1024 x 512 x 16 workload although they move more bytes.
bool adr2d_fused_enabled() {
  const char* e = getenv("RSV_STENCIL_FUSED");
  return e != nullptr && e[0] == '1';
}

template <typename R, int STAGE>
cudaError_t launch_stage(rsv_operator op, const StGeom& g, const R* xin, const R* u, R* acc, const R* f, R* xout,
                         R* ysnap, R h) {
  if (sizeof(R) == 4 && g.nx % 4 == 0) {
    const float* xi = reinterpret_cast<const float*>(xin);
    const float* uu = reinterpret_cast<const float*>(u);
    float* ac = reinterpret_cast<float*>(acc);
    const float* ff = reinterpret_cast<const float*>(f);
    float* xo = reinterpret_cast<float*>(xout);
    float* ys = reinterpret_cast<float*>(ysnap);
    const unsigned gx = (unsigned)((g.nx / 4 + 31) / 32);
    if (op->kind == RSV_OP_ADR2D) {
      dim3 grid(gx, (unsigned)((g.ny + 7) / 8), (unsigned)g.kg);
      adr2d_stage4_kernel<STAGE><<<grid, dim3(32, 8), 0, op->stream>>>(g, xi, uu, ac, ff, xo, ys, (float)h);
    } else {
      const unsigned blocks = gx * (unsigned)((g.ny * g.nz + 7) / 8) * (unsigned)g.kg;
      if (op->bf16_state) {
        // xin, u, xout hold BF16 values at the FP32 slots' addresses
        adv3d_stage4_kernel<STAGE, __nv_bfloat16><<<blocks, dim3(32, 8), 0, op->stream>>>(
            g, reinterpret_cast<const __nv_bfloat16*>(xin), reinterpret_cast<const __nv_bfloat16*>(u), ac, ff,
            reinterpret_cast<__nv_bfloat16*>(xout), ys, (float)h);
      } else {
        adv3d_stage4_kernel<STAGE, float><<<blocks, dim3(32, 8), 0, op->stream>>>(g, xi, uu, ac, ff, xo, ys, (float)h);
      }
    }
    return cudaGetLastError();
  }
  if (op->kind == RSV_OP_ADR2D) {
    dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.kg);
    adr2d_stage_kernel<R, STAGE><<<grid, dim3(32, 8), 0, op->stream>>>(g, xin, u, acc, f, xout, ysnap, h);
  } else {
    dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny * g.nz + 7) / 8), (unsigned)g.kg);
    adv3d_stage_kernel<R, STAGE><<<grid, dim3(32, 8), 0, op->stream>>>(g, xin, u, acc, f, xout, ysnap, h);
  }
  return cudaGetLastError();
}

}  // namespace

// RSV_STENCIL3D_STAGED=1 keeps FP32 3-D marches on the four single-stage kernels (comparisons).
bool adv3d_pairs_enabled() {
  const char* e = getenv("RSV_STENCIL3D_STAGED");
  return !(e != nullptr && e[0] == '1');
}

// RSV_STENCIL2D_STAGED=1 keeps FP32 2-D marches on the four single-stage kernels (comparisons).
bool adr2d_pairs_enabled() {
  static const bool v = [] {
    const char* e = getenv("RSV_STENCIL2D_STAGED");
    return !(e != nullptr && e[0] == '1');
  }();
  return v;
}

// 2-D jet: U(y) = 0.5 (1 + tanh((0.5 - |y|)/delta)), r(y) = -kappa dU/dy, sponge on the fly.
rsv_status build_adr2d(rsv_operator op, const rsv_operator_desc* d) {
  if (d->nx < 3 || d->ny < 3 || !(d->lx > 0) || !(d->ly > 0) || !(d->jet_delta > 0))
    return fail(RSV_ERR_INVALID_ARG, "ADR2D needs nx, ny >= 3 and positive lengths");
  op->nx = d->nx;
  op->ny = d->ny;
  op->nz = 1;
  op->n = (int64_t)d->nx * d->ny;
  op->n_inst = 1;
  op->inst_off.assign(1, 0);
  op->inst_len.assign(1, op->n);
  op->real_state = true;
  op->c_dx = d->lx / (d->nx + 1);
  op->c_dy = d->ly / (d->ny + 1);
  op->visc = d->visc;
  op->sponge_cells = d->sponge_cells;
  op->sponge_amp = d->sponge_amp;
  std::vector<double> U(d->ny), r(d->ny);
  for (int j = 0; j < d->ny; ++j) {
    const double y = -0.5 * d->ly + (j + 1) * op->c_dy;
    const double arg = (0.5 - std::fabs(y)) / d->jet_delta;
    U[j] = 0.5 * (1.0 + std::tanh(arg));
    const double sg = (y > 0) - (y < 0);
    const double ch = std::cosh(arg);
    r[j] = -d->kappa * (0.5 / (ch * ch) * (-sg / d->jet_delta));
  }
  return upload_fields(op, {U, r});
}

// 3-D boundary layer: U = erf(r / delta(x)) and its exact gradient (0 on the axis r = 0).
rsv_status build_adv3d(rsv_operator op, const rsv_operator_desc* d) {
  if (d->nx < 3 || d->ny < 3 || d->nz < 3 || !(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0))
    return fail(RSV_ERR_INVALID_ARG, "ADV3D needs nx, ny, nz >= 3 and positive lengths");
  op->nx = d->nx;
  op->ny = d->ny;
  op->nz = d->nz;
  const int64_t ncell = (int64_t)d->nx * d->ny * d->nz;
  op->n = 3 * ncell;
  op->n_inst = 1;
  op->inst_off.assign(1, 0);
  op->inst_len.assign(1, op->n);
  op->real_state = true;
  op->c_dx = d->lx / (d->nx + 1);
  op->c_dy = d->ly / (d->ny + 1);
  op->c_dz = d->lz / (d->nz + 1);
  op->visc = d->visc;
  std::vector<double> U(ncell), Ux(ncell), Uy(ncell), Uz(ncell);
  const double dd = (d->delta1 - d->delta0) / d->lx;
  for (int kz = 0; kz < d->nz; ++kz)
    for (int j = 0; j < d->ny; ++j)
      for (int i = 0; i < d->nx; ++i) {
        const int64_t q = ((int64_t)kz * d->ny + j) * d->nx + i;
        const double x = (i + 1) * op->c_dx;
        const double y = -0.5 * d->ly + (j + 1) * op->c_dy;
        const double z = -0.5 * d->lz + (kz + 1) * op->c_dz;
        const double del = d->delta0 + dd * x;
        const double r = std::sqrt(y * y + z * z);
        const double gg = 2.0 / std::sqrt(M_PI) * std::exp(-(r / del) * (r / del));
        U[q] = std::erf(r / del);
        Ux[q] = gg * (-r * dd / (del * del));
        Uy[q] = r > 0 ? gg * (y / (r * del)) : 0.0;
        Uz[q] = r > 0 ? gg * (z / (r * del)) : 0.0;
      }
  rsv_status st = upload_fields(op, {U, Ux, Uy, Uz});
  if (st != RSV_OK || op->prec != RSV_PREC_FP32) return st;
  // the pair kernels read the four fields of a cell with one 16-byte load
  std::vector<float> il(4 * U.size());
  for (size_t q = 0; q < U.size(); ++q) {
    il[4 * q] = (float)U[q];
    il[4 * q + 1] = (float)Ux[q];
    il[4 * q + 2] = (float)Uy[q];
    il[4 * q + 3] = (float)Uz[q];
  }
  return upload(op, il.data(), il.size() * sizeof(float), &op->fld[4]);
}

// Workspace behind the state in the march: two stage-input buffers and the accumulator.
size_t stencil_scratch_bytes(rsv_operator op, int kg) {
  return 3 * (size_t)kg * op->n * (op->prec == RSV_PREC_FP64 ? 8 : 4);
}

template <typename R>
cudaError_t stencil_march_tile(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y) {
  const StGeom g = geom_of(op, t.kg, t.adjoint);
  const int64_t rows = (int64_t)t.kg * op->n;
  R* u = static_cast<R*>(state);
  R* xa = u + rows;
  R* xb = xa + rows;
  R* acc = xb + rows;
  const R h = (R)op->h;
  cudaError_t e = cudaSuccess;
  if (op->kind == RSV_OP_ADR2D && adr2d_fused_enabled()) {
    // whole steps, the field ping-pongs between u and xa
    R* cur = u;
    R* nxt = xa;
    for (int s = 0; s < t.steps && e == cudaSuccess; ++s) {
      const int64_t n = t.n0 + s;
      const bool forced = F != nullptr && n < t.n_forced;
      const R* Fr = static_cast<const R*>(F);
      const R* f0 = forced ? Fr + (size_t)(2 * s) * rows : nullptr;
      const R* fh = forced ? Fr + (size_t)(2 * s + 1) * rows : nullptr;
      const R* f1 = forced ? Fr + (size_t)(2 * s + 2) * rows : nullptr;
      R* ys = (Y != nullptr && s >= t.y_first) ? static_cast<R*>(Y) + (size_t)s * rows : nullptr;
      e = launch_adr2d_step<R>(op, g, cur, nxt, f0, fh, f1, ys, h);
      std::swap(cur, nxt);
    }
    if (e == cudaSuccess && cur != u) e = cudaMemcpyAsync(u, cur, sizeof(R) * rows, cudaMemcpyDeviceToDevice, op->stream);
    if (e == cudaSuccess) e = check_finite(op, u, rows, true);
    return e;
  }
  const bool pairs3d = sizeof(R) == 4 && op->kind == RSV_OP_ADV3D && adv3d_pairs_enabled() && !op->bf16_state &&
                       op->nx % 4 == 0 && op->n < ((int64_t)1 << 31);
  const bool pairs2d = sizeof(R) == 4 && op->kind == RSV_OP_ADR2D && adr2d_pairs_enabled() && op->nx % 4 == 0 &&
                       op->n < ((int64_t)1 << 31);
  if (pairs3d || pairs2d) {
    // two fused stage pairs per step; the state ping-pongs between u and xb, x3 lives in xa
    float* cur = reinterpret_cast<float*>(u);
    float* nxt = reinterpret_cast<float*>(xb);
    for (int s = 0; s < t.steps && e == cudaSuccess; ++s) {
      const int64_t n = t.n0 + s;
      const bool forced = F != nullptr && n < t.n_forced;
      const float* Fr = static_cast<const float*>(F);
      Pair3D pa;
      pa.in = cur;
      pa.u = nullptr;
      pa.acc = nullptr;
      pa.fa = forced ? Fr + (size_t)(2 * s) * rows : nullptr;
      pa.fb = forced ? Fr + (size_t)(2 * s + 1) * rows : nullptr;
      pa.out = reinterpret_cast<float*>(xa);
      pa.acc_out = reinterpret_cast<float*>(acc);
      pa.ysnap = (Y != nullptr && s >= t.y_first) ? static_cast<float*>(Y) + (size_t)s * rows : nullptr;
      pa.h = (float)op->h;
      Pair3D pb = pa;
      pb.in = reinterpret_cast<const float*>(xa);
      pb.u = cur;
      pb.acc = reinterpret_cast<const float*>(acc);
      pb.fa = pa.fb;
      pb.fb = forced ? Fr + (size_t)(2 * s + 2) * rows : nullptr;
      pb.out = nxt;
      pb.acc_out = nullptr;
      pb.ysnap = nullptr;
      if (pairs2d) {   // the 2-D kernels take the direction from g.adjoint
        e = launch_pair2d<false>(op, g, pa);
        if (e == cudaSuccess) e = launch_pair2d<true>(op, g, pb);
      } else if (t.adjoint) {
        e = launch_pair3d<true, false>(op, g, pa);
        if (e == cudaSuccess) e = launch_pair3d<true, true>(op, g, pb);
      } else {
        e = launch_pair3d<false, false>(op, g, pa);
        if (e == cudaSuccess) e = launch_pair3d<false, true>(op, g, pb);
      }
      std::swap(cur, nxt);
    }
    if (e == cudaSuccess && cur != reinterpret_cast<float*>(u))
      e = cudaMemcpyAsync(u, cur, sizeof(float) * rows, cudaMemcpyDeviceToDevice, op->stream);
    if (e == cudaSuccess) e = check_finite(op, u, rows, true);
    return e;
  }
  for (int s = 0; s < t.steps && e == cudaSuccess; ++s) {
    const int64_t n = t.n0 + s;
    const bool forced = F != nullptr && n < t.n_forced;
    const R* Fr = static_cast<const R*>(F);
    const R* f0 = forced ? Fr + (size_t)(2 * s) * rows : nullptr;
    const R* fh = forced ? Fr + (size_t)(2 * s + 1) * rows : nullptr;
    const R* f1 = forced ? Fr + (size_t)(2 * s + 2) * rows : nullptr;
    R* ys = (Y != nullptr && s >= t.y_first) ? static_cast<R*>(Y) + (size_t)s * rows : nullptr;
    // stage inputs ping-pong between xa and xb: a stage never writes the array its stencil reads
    e = launch_stage<R, 1>(op, g, u, u, acc, f0, xa, ys, h);
    if (e == cudaSuccess) e = launch_stage<R, 2>(op, g, xa, u, acc, fh, xb, nullptr, h);
    if (e == cudaSuccess) e = launch_stage<R, 3>(op, g, xb, u, acc, fh, xa, nullptr, h);
    if (e == cudaSuccess) e = launch_stage<R, 4>(op, g, xa, nullptr, acc, f1, u, nullptr, h);
  }
  if (e == cudaSuccess) e = check_finite(op, u, rows, true);
  return e;
}

template <typename R>
cudaError_t stencil_apply(rsv_operator op, const void* x, int k, bool adjoint, void* y) {
  // complex blocks: the real operator acts on real and imaginary parts alike (test entry point)
  const StGeom g = geom_of(op, k, adjoint);
  const int64_t count = (int64_t)k * op->n;
  R* tmp = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&tmp, 4 * count * sizeof(R), op->stream);
  if (e != cudaSuccess) return e;
  const unsigned b = (unsigned)((count + 255) / 256);
  split_kernel<R><<<b, 256, 0, op->stream>>>((const cpx<R>*)x, count, tmp, tmp + count);
  for (int part = 0; part < 2; ++part) {
    if (op->kind == RSV_OP_ADR2D) {
      dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)k);
      adr2d_apply_real_kernel<R><<<grid, dim3(32, 8), 0, op->stream>>>(g, tmp + part * count, tmp + (2 + part) * count);
    } else {
      dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny * g.nz + 7) / 8), (unsigned)k);
      adv3d_apply_real_kernel<R><<<grid, dim3(32, 8), 0, op->stream>>>(g, tmp + part * count, tmp + (2 + part) * count);
    }
  }
  join_kernel<R><<<b, 256, 0, op->stream>>>(tmp + 2 * count, tmp + 3 * count, count, (cpx<R>*)y);
  e = cudaGetLastError();
  cudaFreeAsync(tmp, op->stream);
  return e;
}

template cudaError_t stencil_march_tile<double>(rsv_operator, const MarchTile&, void*, const void*, void*);
template cudaError_t stencil_march_tile<float>(rsv_operator, const MarchTile&, void*, const void*, void*);
template cudaError_t stencil_apply<double>(rsv_operator, const void*, int, bool, void*);
template cudaError_t stencil_apply<float>(rsv_operator, const void*, int, bool, void*);

}  // namespace rsv
