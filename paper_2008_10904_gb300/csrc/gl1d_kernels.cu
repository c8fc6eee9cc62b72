// RK4 and Crank-Nicolson marches of 1-D three-point (tridiagonal) operators: the linearised
// Ginzburg-Landau family of Sec. 3, Eq. (GL_timeDomain), discretised with
// central differences, one or many independent instances.
//
// One CTA owns one (instance, test vector) pair for a whole time tile: the
// state lives in registers (PPT points per thread), each RK4 stage
// exchanges the stage input through shared memory (one barrier per stage,
// two alternating buffers), and the forcing for the tile's 2S+1 stage times
// is read from the synthesis tile F.  The state at the start of each
// analysed step is written to the snapshot tile Y for the analysis kernel.
//
//   k1 = A u + f(t_n)
//   k2 = A (u + h/2 k1) + f(t_n + h/2)
//   k3 = A (u + h/2 k2) + f(t_n + h/2)
//   k4 = A (u + h k3)   + f(t_n + h)
//   u <- u + h/6 (k1 + 2 k2 + 2 k3 + k4)
#include "rsv_internal.h"

namespace rsv {
namespace {

template <typename R, int PPT, int MAXT>
__global__ void __launch_bounds__(MAXT) gl1d_tile_kernel(Gl1dTile t, cpx<R>* __restrict__ u,
                                                         const cpx<R>* __restrict__ F, cpx<R>* __restrict__ Y,
                                                         double* __restrict__ norms, int* __restrict__ flag) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.x;
  const int v = blockIdx.y;
  const int64_t off = t.inst_off[inst];
  const int len = (int)(t.inst_off[inst + 1] - off);
  const int ld = t.max_n + 2;
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][max_n + 2], zero halo at both ends
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R> zero = mk<R>(0, 0);
  if (threadIdx.x == 0) {
    sx[0] = zero;
    sx[ld] = zero;
    sx[len + 1] = zero;
    sx[ld + len + 1] = zero;
  }
  const int64_t rows = (int64_t)t.kg * t.n;
  const int64_t rbase = (int64_t)v * t.n + off;
  cpx<R> cl[PPT], cd[PPT], cu[PPT], us[PPT];
  bool ok[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int i = threadIdx.x + m * blockDim.x;
    ok[m] = i < len;
    if (ok[m]) {
      cl[m] = lo[off + i];
      cd[m] = di[off + i];
      cu[m] = up[off + i];
      us[m] = u[rbase + i];
    } else {
      cl[m] = cd[m] = cu[m] = us[m] = zero;
    }
  }
  const R h = R(t.h);
  const R h2 = R(0.5) * h;
  const R h6 = h / R(6);
  int buf = 0;
  // y = A x + f for the owned points; x is written to the shared buffer first.
  auto stage = [&](const cpx<R>* x, const cpx<R>* f, cpx<R>* y) {
    cpx<R>* s = sx + buf * ld;
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (ok[m]) s[1 + threadIdx.x + m * blockDim.x] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int i = threadIdx.x + m * blockDim.x;
      cpx<R> a = f[m];
      if (ok[m]) {
        cfma(a, cl[m], s[i]);
        cfma(a, cd[m], x[m]);
        cfma(a, cu[m], s[i + 2]);
      }
      y[m] = a;
    }
    buf ^= 1;
  };
  // Forcing of step s: f(t_n + h/2) and f(t_n + h); f(t_n) is the previous
  // step's f(t_n + h).  The loads for step s + 1 are issued at the start of
  // step s, so their latency overlaps the step.
  auto load_f = [&](int s, cpx<R>* fh_out, cpx<R>* f1_out) {
    const bool forced = (F != nullptr) && (t.n0 + s < t.n_forced);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      fh_out[m] = f1_out[m] = zero;
      if (forced && ok[m]) {
        const int64_t r = rbase + threadIdx.x + m * blockDim.x;
        fh_out[m] = F[(int64_t)(2 * s + 1) * rows + r];
        f1_out[m] = F[(int64_t)(2 * s + 2) * rows + r];
      }
    }
  };
  cpx<R> f0[PPT], fh[PPT], f1[PPT], nfh[PPT], nf1[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) f0[m] = nfh[m] = nf1[m] = zero;
  if (F != nullptr && t.n0 < t.n_forced) {
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (ok[m]) f0[m] = F[rbase + threadIdx.x + m * blockDim.x];
  }
  load_f(0, fh, f1);
  for (int s = 0; s < t.steps; ++s) {
    if (s + 1 < t.steps) load_f(s + 1, nfh, nf1);
    if (!((F != nullptr) && (t.n0 + s < t.n_forced))) {
#pragma unroll
      for (int m = 0; m < PPT; ++m) f0[m] = zero;   // unforced steps carry no forcing at any stage
    }
    if (Y != nullptr && s >= t.y_first) {
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (ok[m]) Y[(int64_t)s * rows + rbase + threadIdx.x + m * blockDim.x] = us[m];
    }
    // k1 + 2 k2 + 2 k3 accumulates in acc; x is the next stage input
    cpx<R> k[PPT], x[PPT], acc[PPT];
    stage(us, f0, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = k[m];
      x[m] = us[m] + h2 * k[m];
    }
    stage(x, fh, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h2 * k[m];
    }
    stage(x, fh, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h * k[m];
    }
    stage(x, f1, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      us[m] = us[m] + h6 * (acc[m] + k[m]);
      f0[m] = f1[m];
      fh[m] = nfh[m];
      f1[m] = nf1[m];
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    if (ok[m]) {
      u[rbase + threadIdx.x + m * blockDim.x] = us[m];
      nrm += (double)us[m].re * (double)us[m].re + (double)us[m].im * (double)us[m].im;
    }
  }
  // block reduction of |u|^2 for the norm monitor
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    if (norms != nullptr) norms[(int64_t)v * t.n_inst + inst] = tot;
    if (!(tot < 1e300)) atomicExch(flag, 1);  // NaN or overflow
  }
}

// Crank-Nicolson tile kernel (the time scheme of the paper's Sec. 3 case):
//   (I - h/2 A) u_{n+1} = (I + h/2 A) u_n + h/2 (f(t_n) + f(t_n + h)).
// The right-hand side d is formed in registers (one neighbour exchange through shared memory);
// the constant tridiagonal system is solved by parallel cyclic reduction: at level l (distance
// s = 2^l) every point eliminates its neighbours at -s and +s,
//   d_i <- d_i - cl_i^l d_{i-s} - cu_i^l d_{i+s},
// with factors cl, cu precomputed in FP64 on the host for the step h, and after
// ceil(log2 max_n) levels u_i = d_i / b_i (inverse pivots precomputed too).  One barrier per level.
template <typename R, int PPT, int MAXT>
__global__ void __launch_bounds__(MAXT) gl1d_cn_tile_kernel(Gl1dTile t, cpx<R>* __restrict__ u,
                                                            const cpx<R>* __restrict__ F, cpx<R>* __restrict__ Y,
                                                            double* __restrict__ norms, int* __restrict__ flag) {
  extern __shared__ unsigned char smem_raw[];
  const int inst = blockIdx.x;
  const int v = blockIdx.y;
  const int64_t off = t.inst_off[inst];
  const int len = (int)(t.inst_off[inst + 1] - off);
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][max_n]
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R>* cl = reinterpret_cast<const cpx<R>*>(t.cr_lo);
  const cpx<R>* cu = reinterpret_cast<const cpx<R>*>(t.cr_up);
  const cpx<R>* inv = reinterpret_cast<const cpx<R>*>(t.cr_inv);
  const cpx<R> zero = mk<R>(0, 0);
  const int64_t rows = (int64_t)t.kg * t.n;
  const int64_t rbase = (int64_t)v * t.n + off;
  cpx<R> clo[PPT], cdi[PPT], cup[PPT], us[PPT], pinv[PPT];
  bool ok[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int i = threadIdx.x + m * blockDim.x;
    ok[m] = i < len;
    clo[m] = cdi[m] = cup[m] = us[m] = pinv[m] = zero;
    if (ok[m]) {
      clo[m] = lo[off + i];
      cdi[m] = di[off + i];
      cup[m] = up[off + i];
      pinv[m] = inv[off + i];
      us[m] = u[rbase + i];
    }
  }
  const R hh = R(0.5) * R(t.h);
  int buf = 0;
  cpx<R> f0[PPT], f1[PPT];
  const bool forced0 = F != nullptr && t.n0 < t.n_forced;
#pragma unroll
  for (int m = 0; m < PPT; ++m) f0[m] = (forced0 && ok[m]) ? F[rbase + threadIdx.x + m * blockDim.x] : zero;
  for (int s = 0; s < t.steps; ++s) {
    const bool forced = F != nullptr && t.n0 + s < t.n_forced;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      f1[m] = (forced && ok[m]) ? F[(int64_t)(2 * s + 2) * rows + rbase + threadIdx.x + m * blockDim.x] : zero;
      if (!forced) f0[m] = zero;
    }
    if (Y != nullptr && s >= t.y_first) {
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (ok[m]) Y[(int64_t)s * rows + rbase + threadIdx.x + m * blockDim.x] = us[m];
    }
    // d = u + h/2 (A u + f0 + f1)
    cpx<R>* sb = sx + buf * t.max_n;
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (ok[m]) sb[threadIdx.x + m * blockDim.x] = us[m];
    __syncthreads();
    cpx<R> d[PPT];
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int i = threadIdx.x + m * blockDim.x;
      cpx<R> a = f0[m] + f1[m];
      if (ok[m]) {
        if (i > 0) cfma(a, clo[m], sb[i - 1]);
        cfma(a, cdi[m], us[m]);
        if (i + 1 < len) cfma(a, cup[m], sb[i + 1]);
      }
      d[m] = ok[m] ? us[m] + hh * a : zero;
    }
    buf ^= 1;
    // cyclic reduction of (I - h/2 A) u' = d
    for (int l = 0; l < t.cr_levels; ++l) {
      const int sd = 1 << l;
      cpx<R>* sl = sx + buf * t.max_n;
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (ok[m]) sl[threadIdx.x + m * blockDim.x] = d[m];
      __syncthreads();
#pragma unroll
      for (int m = 0; m < PPT; ++m) {
        const int i = threadIdx.x + m * blockDim.x;
        if (!ok[m]) continue;
        const int64_t k = (int64_t)l * t.n + off + i;
        cpx<R> r = d[m];
        if (i - sd >= 0) r = r - cl[k] * sl[i - sd];
        if (i + sd < len) r = r - cu[k] * sl[i + sd];
        d[m] = r;
      }
      buf ^= 1;
    }
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      us[m] = pinv[m] * d[m];
      f0[m] = f1[m];
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    if (ok[m]) {
      u[rbase + threadIdx.x + m * blockDim.x] = us[m];
      nrm += (double)us[m].re * (double)us[m].re + (double)us[m].im * (double)us[m].im;
    }
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    if (norms != nullptr) norms[(int64_t)v * t.n_inst + inst] = tot;
    if (!(tot < 1e300)) atomicExch(flag, 1);
  }
}

// Packed RK4 tile kernel for batches of uneven instances: one CTA of PPT x blockDim slots holds
// several (instance, vector) segments back to back, each followed by a zero slot, so the three-point
// stencil of a segment's end points reads zeros exactly as at an instance's Dirichlet ends.
// map[pack][slot] is the row (vector * n + point) of the slot's point, or -1 for a separator or an
// unused slot.  The steps, the stage exchange and the forcing prefetch are those of
// gl1d_tile_kernel; the divergence flag is raised per point (the march reads norms elsewhere).
template <typename R, int PPT>
__global__ void __launch_bounds__(1024) gl1d_pack_kernel(Gl1dTile t, const int32_t* __restrict__ map,
                                                         cpx<R>* __restrict__ u, const cpx<R>* __restrict__ F,
                                                         cpx<R>* __restrict__ Y, int* __restrict__ flag) {
  extern __shared__ unsigned char smem_raw[];
  const int cap = PPT * (int)blockDim.x;
  const int ld = cap + 2;
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][cap + 2]: zero halo, slots 1..cap, zero
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R> zero = mk<R>(0, 0);
  for (int i = threadIdx.x; i < 2 * ld; i += blockDim.x) sx[i] = zero;   // separators stay zero
  const int64_t rows = (int64_t)t.kg * t.n;
  const int32_t* pm = map + (int64_t)blockIdx.x * cap;
  int64_t row[PPT];
  cpx<R> cl[PPT], cd[PPT], cu[PPT], us[PPT];
  bool ok[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int i = threadIdx.x + m * blockDim.x;
    const int32_t r = pm[i];
    ok[m] = r >= 0;
    row[m] = r;
    if (ok[m]) {
      const int64_t p = r % t.n;
      cl[m] = lo[p];
      cd[m] = di[p];
      cu[m] = up[p];
      us[m] = u[r];
    } else {
      cl[m] = cd[m] = cu[m] = us[m] = zero;
    }
  }
  __syncthreads();
  const R h = R(t.h);
  const R h2 = R(0.5) * h;
  const R h6 = h / R(6);
  int buf = 0;
  auto stage = [&](const cpx<R>* x, const cpx<R>* f, cpx<R>* y) {
    cpx<R>* s = sx + buf * ld;
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (ok[m]) s[1 + threadIdx.x + m * blockDim.x] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int i = threadIdx.x + m * blockDim.x;
      cpx<R> a = f[m];
      if (ok[m]) {
        cfma(a, cl[m], s[i]);
        cfma(a, cd[m], x[m]);
        cfma(a, cu[m], s[i + 2]);
      }
      y[m] = a;
    }
    buf ^= 1;
  };
  auto load_f = [&](int s, cpx<R>* fh_out, cpx<R>* f1_out) {
    const bool forced = (F != nullptr) && (t.n0 + s < t.n_forced);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      fh_out[m] = f1_out[m] = zero;
      if (forced && ok[m]) {
        fh_out[m] = F[(int64_t)(2 * s + 1) * rows + row[m]];
        f1_out[m] = F[(int64_t)(2 * s + 2) * rows + row[m]];
      }
    }
  };
  cpx<R> f0[PPT], fh[PPT], f1[PPT], nfh[PPT], nf1[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) f0[m] = nfh[m] = nf1[m] = zero;
  if (F != nullptr && t.n0 < t.n_forced) {
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (ok[m]) f0[m] = F[row[m]];
  }
  load_f(0, fh, f1);
  for (int s = 0; s < t.steps; ++s) {
    if (s + 1 < t.steps) load_f(s + 1, nfh, nf1);
    if (!((F != nullptr) && (t.n0 + s < t.n_forced))) {
#pragma unroll
      for (int m = 0; m < PPT; ++m) f0[m] = zero;
    }
    if (Y != nullptr && s >= t.y_first) {
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (ok[m]) Y[(int64_t)s * rows + row[m]] = us[m];
    }
    cpx<R> k[PPT], x[PPT], acc[PPT];
    stage(us, f0, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = k[m];
      x[m] = us[m] + h2 * k[m];
    }
    stage(x, fh, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h2 * k[m];
    }
    stage(x, fh, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h * k[m];
    }
    stage(x, f1, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      us[m] = us[m] + h6 * (acc[m] + k[m]);
      f0[m] = f1[m];
      fh[m] = nfh[m];
      f1[m] = nf1[m];
    }
  }
  bool bad = false;
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    if (ok[m]) {
      u[row[m]] = us[m];
      const double q = (double)us[m].re * (double)us[m].re + (double)us[m].im * (double)us[m].im;
      bad = bad || !(q < 1e300);
    }
  }
  if (bad) atomicExch(flag, 1);   // NaN or overflow
}

template <typename R>
__global__ void gl1d_apply_kernel(Gl1dTile t, const cpx<R>* __restrict__ x, cpx<R>* __restrict__ y,
                                  const int32_t* __restrict__ inst_of_point) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (p >= t.n) return;
  const int inst = inst_of_point[p];
  const int64_t a = t.inst_off[inst], b = t.inst_off[inst + 1];
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R>* xv = x + (int64_t)v * t.n;
  cpx<R> acc = mk<R>(0, 0);
  if (p > a) cfma(acc, lo[p], xv[p - 1]);
  cfma(acc, di[p], xv[p]);
  if (p + 1 < b) cfma(acc, up[p], xv[p + 1]);
  y[(int64_t)v * t.n + p] = acc;
}

template <typename R, int PPT, int MAXT>
cudaError_t launch_ppt(const Gl1dTile& t, int threads, void* u, const void* F, void* Y, double* norms, int* flag,
                       cudaStream_t st) {
  const size_t smem = sizeof(cpx<R>) * 2 * (size_t)(t.max_n + 2);
  dim3 grid((unsigned)t.n_inst, (unsigned)t.kg);
  if (t.cr_levels > 0) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(gl1d_cn_tile_kernel<R, PPT, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gl1d_cn_tile_kernel<R, PPT, MAXT><<<grid, threads, smem, st>>>(t, (cpx<R>*)u, (const cpx<R>*)F, (cpx<R>*)Y,
                                                                    norms, flag);
    return cudaGetLastError();
  }
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(gl1d_tile_kernel<R, PPT, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gl1d_tile_kernel<R, PPT, MAXT><<<grid, threads, smem, st>>>(t, (cpx<R>*)u, (const cpx<R>*)F, (cpx<R>*)Y, norms,
                                                               flag);
  return cudaGetLastError();
}

}  // namespace

// One CTA per (instance, vector); PPT points per thread, interleaved (point
// i = thread + m * blockDim) so that every load and store is coalesced.
template <typename R>
cudaError_t launch_gl1d_tile(const Gl1dTile& t, void* u, const void* F, void* Y, double* norms, int* flag,
                             cudaStream_t st) {
  if (t.max_n > 4096) return cudaErrorInvalidValue;
  const int ppt = t.max_n <= 1024 ? 1 : (t.max_n <= 2048 ? 2 : 4);
  const int threads = (((t.max_n + ppt - 1) / ppt + 31) / 32) * 32;
  if (ppt == 1) return launch_ppt<R, 1, 1024>(t, threads, u, F, Y, norms, flag, st);
  if (ppt == 2) return launch_ppt<R, 2, 1024>(t, threads, u, F, Y, norms, flag, st);
  return launch_ppt<R, 4, 1024>(t, threads, u, F, Y, norms, flag, st);
}

// Packed launch: n_packs CTAs of 1024 threads, ppt slots per thread (map from build_gl1d_packs).
template <typename R>
cudaError_t launch_gl1d_pack(const Gl1dTile& t, const int32_t* map, int n_packs, int ppt, void* u, const void* F,
                             void* Y, int* flag, cudaStream_t st) {
  const int threads = 1024;
  const size_t smem = sizeof(cpx<R>) * 2 * (size_t)(ppt * threads + 2);
  auto go = [&](auto kernel) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kernel<<<(unsigned)n_packs, threads, smem, st>>>(t, map, (cpx<R>*)u, (const cpx<R>*)F, (cpx<R>*)Y, flag);
    return cudaGetLastError();
  };
  if (ppt == 1) return go(gl1d_pack_kernel<R, 1>);
  if (ppt == 2) return go(gl1d_pack_kernel<R, 2>);
  if (ppt == 3) return go(gl1d_pack_kernel<R, 3>);
  if (ppt == 4) return go(gl1d_pack_kernel<R, 4>);
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_gl1d_apply(const Gl1dTile& t, const int32_t* inst_of_point, const void* x, void* y,
                              cudaStream_t st) {
  dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)t.kg);
  gl1d_apply_kernel<R><<<grid, 256, 0, st>>>(t, (const cpx<R>*)x, (cpx<R>*)y, inst_of_point);
  return cudaGetLastError();
}

template cudaError_t launch_gl1d_tile<double>(const Gl1dTile&, void*, const void*, void*, double*, int*,
                                             cudaStream_t);
template cudaError_t launch_gl1d_tile<float>(const Gl1dTile&, void*, const void*, void*, double*, int*,
                                            cudaStream_t);
template cudaError_t launch_gl1d_pack<double>(const Gl1dTile&, const int32_t*, int, int, void*, const void*, void*,
                                             int*, cudaStream_t);
template cudaError_t launch_gl1d_pack<float>(const Gl1dTile&, const int32_t*, int, int, void*, const void*, void*,
                                            int*, cudaStream_t);
template cudaError_t launch_gl1d_apply<double>(const Gl1dTile&, const int32_t*, const void*, void*, cudaStream_t);
template cudaError_t launch_gl1d_apply<float>(const Gl1dTile&, const int32_t*, const void*, void*, cudaStream_t);

}  // namespace rsv
