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
#include <cooperative_groups.h>

#include <mutex>

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

// RK4 tile kernel for a few long FP64 marches (fewer (instance, vector) pairs than SMs): one
// thread-block cluster of CS CTAs per pair, each CTA owning a contiguous chunk of ch = ceil(len / CS) of
// the instance's points, so that the FP64 arithmetic of one march (the limit of the one-CTA kernel:
// FP64 runs at a small fraction of the FP32 rate) is spread over CS SMs.  A cluster barrier costs far
// more than a CTA barrier, so there is one per M steps, not one per stage: every M steps each CTA
// publishes its chunk's state in shared memory, and after the cluster barrier reads the H = 4 M points
// beyond each end of its chunk from the CTAs that own them (distributed shared memory).  It then takes
// M steps of four RK4 stages on the widened range [-H, ch + H) with CTA barriers only: a stage is
// exact wherever its input is exact at the point and both neighbours, so the exact range shrinks by
// one point per side and stage and after 4 M stages still covers the chunk.  Points outside the
// instance have zero coefficients, forcing and state, and stay zero (the Dirichlet ends).  Every CTA of a
// cluster, including one that owns no point, runs the same sequence of cluster barriers; the last one
// keeps each CTA resident until the other CTAs' reads of its shared memory are done.
template <typename R, int CS, int M>
__global__ void gl1d_cluster_kernel(Gl1dTile t, cpx<R>* __restrict__ u, const cpx<R>* __restrict__ F,
                                    cpx<R>* __restrict__ Y, double* __restrict__ norms, int* __restrict__ flag) {
  namespace cg = cooperative_groups;
  constexpr int kHalo = 4 * M;                    // points of the widened range beyond each chunk end
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ double part;
  const int rank = (int)cluster.block_rank();
  const int inst = blockIdx.x / CS;
  const int v = blockIdx.y;
  const int64_t off = t.inst_off[inst];
  const int len = (int)(t.inst_off[inst + 1] - off);
  const int ch = (len + CS - 1) / CS;            // points per CTA of this instance
  const int p0 = rank * ch;                       // first point of this CTA
  const int cnt = max(0, min(ch, len - p0));      // points it owns (the last CTAs may own fewer or none)
  const int nt = (int)blockDim.x;                 // >= ch_max + 2 kHalo
  const int pub = nt - 2 * kHalo;                 // >= the longest chunk
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][nt + 2]: position e at slot 1 + e
  cpx<R>* ush = sx + 2 * (nt + 2);                  // [2][pub]: the chunk's state, published per step
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R> zero = mk<R>(0, 0);
  const int e = threadIdx.x;                      // position on the widened range
  const int j = e - kHalo;                        // point index relative to the chunk
  const int q = p0 + j;                           // point index in the instance
  const bool inside = j < ch + kHalo && q >= 0 && q < len;
  const bool owned = j >= 0 && j < cnt;
  const int64_t rows = (int64_t)t.kg * t.n;
  const int64_t r = (int64_t)v * t.n + off + q;   // this position's row (when inside)
  // owner of a halo point and its slot in the owner's published chunk
  const cpx<R>* halo_src = nullptr;
  if (inside && !owned) halo_src = cluster.map_shared_rank(ush, q / ch) + q % ch;
  cpx<R> cl = zero, cd = zero, cu = zero, us = zero;
  if (inside) {
    cl = lo[off + q];
    cd = di[off + q];
    cu = up[off + q];
  }
  if (owned) us = u[r];
  for (int i = threadIdx.x; i < 2 * (nt + 2); i += nt) sx[i] = zero;   // the range's outer slots stay zero
  __syncthreads();
  const R h = R(t.h);
  const R h2 = R(0.5) * h;
  const R h6 = h / R(6);
  int buf = 0;
  // y = A x + f on the widened range (CTA barrier; the range's ends read zero)
  auto stage = [&](const cpx<R>& x, const cpx<R>& f) -> cpx<R> {
    cpx<R>* s = sx + buf * (nt + 2);
    s[1 + e] = x;
    __syncthreads();
    cpx<R> a = f;
    cfma(a, cl, s[e]);
    cfma(a, cd, x);
    cfma(a, cu, s[e + 2]);
    buf ^= 1;
    return a;
  };
  auto forced = [&](int s) { return F != nullptr && t.n0 + s < t.n_forced; };
  cpx<R> f0 = zero, fh = zero, f1 = zero, nfh = zero, nf1 = zero;
  if (inside && forced(0)) {
    f0 = F[r];
    fh = F[rows + r];
    f1 = F[2 * rows + r];
  }
  for (int s = 0; s < t.steps; ++s) {
    if (inside && s + 1 < t.steps && forced(s + 1)) {   // next step's forcing, in flight during this step
      nfh = F[(int64_t)(2 * s + 3) * rows + r];
      nf1 = F[(int64_t)(2 * s + 4) * rows + r];
    }
    if (!forced(s)) f0 = fh = f1 = zero;
    if (owned && Y != nullptr && s >= t.y_first) Y[(int64_t)s * rows + r] = us;
    if (s % M == 0) {   // publish the chunk's state, then take the halo's from its owners
      const int b = (s / M) & 1;
      if (owned) ush[b * pub + j] = us;
      cluster.sync();
      if (halo_src != nullptr) us = halo_src[b * pub];
    }
    cpx<R> k = stage(us, f0);
    cpx<R> acc = k;
    k = stage(us + h2 * k, fh);
    acc = acc + R(2) * k;
    k = stage(us + h2 * k, fh);
    acc = acc + R(2) * k;
    k = stage(us + h * k, f1);
    us = inside ? us + h6 * (acc + k) : zero;   // the halo evolves too until the next exchange
    f0 = f1;
    fh = nfh;
    f1 = nf1;
  }
  double nrm = 0.0;
  if (owned) {
    u[r] = us;
    nrm = (double)us.re * (double)us.re + (double)us.im * (double)us.im;
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < nt / 32; ++w) tot += red[w];
    part = tot;
  }
  cluster.sync();
  if (rank == 0 && threadIdx.x == 0) {
    double tot = 0.0;
    for (int c = 0; c < CS; ++c) tot += *cluster.map_shared_rank(&part, c);
    if (norms != nullptr) norms[(int64_t)v * t.n_inst + inst] = tot;
    if (!(tot < 1e300)) atomicExch(flag, 1);  // NaN or overflow
  }
  cluster.sync();
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

// Packed RK4 tile kernel for batches of uneven instances: one CTA of NT threads x PPT slots holds
// several (instance, vector) segments back to back, each followed by a zero slot, so the three-point
// stencil of a segment's end points reads zeros exactly as at an instance's Dirichlet ends.
// map[pack][slot] is the row (vector * n + point) of the slot's point, or -1 for a separator or an
// unused slot; slot i = thread + m * NT.  The state stays in registers and each stage exchanges its
// input through shared memory, as in gl1d_tile_kernel.  The forcing at t_n + h/2 and t_n + h is copied
// into a shared-memory ring RING - 1 steps ahead of its use (cp.async, issued and waited for by the
// thread that reads it, so neither registers nor a barrier are spent on it); the forcing at t_n is the
// previous step's t_n + h value, kept in a register.  The divergence flag is raised per point (the
// march reads norms elsewhere).
template <typename R>
__device__ __forceinline__ void cp_async_cpx(cpx<R>* dst, const cpx<R>* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(sizeof(cpx<R>))
               : "memory");
}

template <typename R, int NT, int PPT, int RING>
__global__ void __launch_bounds__(NT, 1) gl1d_pack_kernel(Gl1dTile t, const int32_t* __restrict__ map,
                                                            cpx<R>* __restrict__ u, const cpx<R>* __restrict__ F,
                                                            cpx<R>* __restrict__ Y, int* __restrict__ flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int cap = NT * PPT;
  constexpr int ld = cap + 2;
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][cap + 2]: zero halo, slots 1..cap, zero
  cpx<R>* ring = sx + 2 * ld;                        // [RING][2][cap]: f(t_n + h/2), f(t_n + h)
  const cpx<R>* lo = reinterpret_cast<const cpx<R>*>(t.lo);
  const cpx<R>* di = reinterpret_cast<const cpx<R>*>(t.di);
  const cpx<R>* up = reinterpret_cast<const cpx<R>*>(t.up);
  const cpx<R> zero = mk<R>(0, 0);
  for (int i = threadIdx.x; i < 2 * ld; i += NT) sx[i] = zero;   // separators stay zero
  const int rows = t.kg * (int)t.n;                               // < 2^31 (checked by the host)
  const bool has_f = F != nullptr;
  const int32_t* pm = map + (int64_t)blockIdx.x * cap;
  int32_t row[PPT];
  cpx<R> cl[PPT], cd[PPT], cu[PPT], us[PPT], f0[PPT];
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int32_t r = pm[threadIdx.x + m * NT];
    row[m] = r;
    cl[m] = cd[m] = cu[m] = us[m] = f0[m] = zero;
    if (r >= 0) {
      const int p = r % (int)t.n;
      cl[m] = lo[p];
      cd[m] = di[p];
      cu[m] = up[p];
      us[m] = u[r];
      if (has_f && t.n0 < t.n_forced) f0[m] = F[r];
    }
  }
  // copies of step s's forcing into ring entry s % RING, one commit group per step (empty when the
  // step is unforced or beyond the tile, so that the group count stays one per step)
  auto prefetch = [&](int s) {
    if (s < t.steps && has_f && t.n0 + s < t.n_forced) {
      cpx<R>* dst = ring + (s % RING) * 2 * cap + threadIdx.x;
      const cpx<R>* src = F + (int64_t)(2 * s + 1) * rows;
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (row[m] >= 0) {
          cp_async_cpx(dst + m * NT, src + row[m]);
          cp_async_cpx(dst + cap + m * NT, src + rows + row[m]);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int s = 0; s < RING - 1; ++s) prefetch(s);
  __syncthreads();
  const R h = R(t.h);
  const R h2 = R(0.5) * h;
  const R h6 = h / R(6);
  int buf = 0;
  auto stage = [&](const cpx<R>* x, const cpx<R>* f, cpx<R>* y) {
    cpx<R>* s = sx + buf * ld;
#pragma unroll
    for (int m = 0; m < PPT; ++m)
      if (row[m] >= 0) s[1 + threadIdx.x + m * NT] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int i = threadIdx.x + m * NT;
      cpx<R> a = f[m];
      if (row[m] >= 0) {
        cfma(a, cl[m], s[i]);
        cfma(a, cd[m], x[m]);
        cfma(a, cu[m], s[i + 2]);
      }
      y[m] = a;
    }
    buf ^= 1;
  };
  for (int s = 0; s < t.steps; ++s) {
    prefetch(s + RING - 1);   // into the entry of step s - 1, whose values are already in registers
    asm volatile("cp.async.wait_group %0;" ::"n"(RING - 1) : "memory");   // this thread's step-s copies landed
    const bool fs = has_f && t.n0 + s < t.n_forced;
    const cpx<R>* rh = ring + (s % RING) * 2 * cap + threadIdx.x;
    const cpx<R>* r1 = rh + cap;
    if (Y != nullptr && s >= t.y_first) {
#pragma unroll
      for (int m = 0; m < PPT; ++m)
        if (row[m] >= 0) Y[(int64_t)s * rows + row[m]] = us[m];
    }
    cpx<R> f[PPT], k[PPT], x[PPT], acc[PPT];
#pragma unroll
    for (int m = 0; m < PPT; ++m) f[m] = fs ? f0[m] : zero;
    stage(us, f, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = k[m];
      x[m] = us[m] + h2 * k[m];
      f[m] = fs ? rh[m * NT] : zero;
    }
    stage(x, f, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h2 * k[m];
      f[m] = fs ? rh[m * NT] : zero;
    }
    stage(x, f, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      acc[m] = acc[m] + R(2) * k[m];
      x[m] = us[m] + h * k[m];
      f[m] = fs ? r1[m * NT] : zero;
    }
    stage(x, f, k);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      us[m] = us[m] + h6 * (acc[m] + k[m]);
      f0[m] = f[m];
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // the trailing (empty) groups
  bool bad = false;
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    if (row[m] >= 0) {
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

// One cluster of CS CTAs per (instance, vector), one point per thread.
template <typename R, int CS, int M>
cudaError_t launch_cluster(const Gl1dTile& t, void* u, const void* F, void* Y, double* norms, int* flag,
                           cudaStream_t st) {
  const int chunk = (t.max_n + CS - 1) / CS;
  const int threads = (chunk + 8 * M + 31) / 32 * 32;   // the widened range of the longest chunk
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CS * t.n_inst), (unsigned)t.kg);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = sizeof(cpx<R>) * (2 * (size_t)(threads + 2) + 2 * (size_t)(threads - 8 * M));
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gl1d_cluster_kernel<R, CS, M>, t, (cpx<R>*)u, (const cpx<R>*)F, (cpx<R>*)Y, norms,
                            flag);
}

}  // namespace

// Clusters of 16 CTAs exceed the portable size of 8: taken when the kernel may opt in and the device
// can hold one (asked once per device; a refusal is cleared so no later call reads it as its own).
static bool cluster16_ok(int dev) {
  static std::mutex mu;
  static int state[64] = {0};   // 0 not asked, 1 yes, 2 no
  if (dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lock(mu);
  if (state[dev] == 0) {
    auto kernel = gl1d_cluster_kernel<double, 16, 2>;
    bool ok = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    if (ok) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(32);
      cfg.dynamicSmemBytes = sizeof(cpx<double>) * (2 * 34 + 2 * 16);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      ok = cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) == cudaSuccess && clusters > 0;
    }
    if (!ok) cudaGetLastError();
    state[dev] = ok ? 1 : 2;
  }
  return state[dev] == 1;
}

// Cluster size for the FP64 RK4 march (0: one CTA per pair), such that every (instance, vector) pair's
// cluster fits in one wave.  16 CTAs exchanging every 2 steps when each CTA's chunk and its 8-point
// halos fill one warp (instances of 128 to 256 points): a cluster barrier per two steps and no second,
// mostly idle warp, whose FP64 work costs as much as a full one's.  Otherwise the largest of 8, 4, 2
// for which every CTA of the longest instance owns 32 to 256 points, exchanging every step.
// RSV_GL1D_CLUSTER=0 keeps one CTA per pair.
int gl1d_cluster_size(const Gl1dTile& t) {
  static const bool env = [] {
    const char* e = getenv("RSV_GL1D_CLUSTER");
    return !(e != nullptr && e[0] == '0');
  }();
  if (!env || t.cr_levels > 0) return 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  if (t.max_n >= 128 && t.max_n <= 256 && (int64_t)t.n_inst * t.kg * 16 <= sms && cluster16_ok(dev)) return 16;
  for (int cs = 8; cs >= 2; cs /= 2)
    if (t.max_n >= 32 * cs && (t.max_n + cs - 1) / cs <= 256 && (int64_t)t.n_inst * t.kg * cs <= sms) return cs;
  return 0;
}

// One CTA per (instance, vector); PPT points per thread, interleaved (point
// i = thread + m * blockDim) so that every load and store is coalesced.  FP64
// marches of few pairs take a cluster of CTAs per pair instead.
template <typename R>
cudaError_t launch_gl1d_tile(const Gl1dTile& t, void* u, const void* F, void* Y, double* norms, int* flag,
                             cudaStream_t st) {
  if (t.max_n > 4096) return cudaErrorInvalidValue;
  if constexpr (sizeof(R) == 8) {   // FP64: spread each march over a cluster of SMs when there are few
    const int cs = gl1d_cluster_size(t);
    if (cs == 16) return launch_cluster<R, 16, 2>(t, u, F, Y, norms, flag, st);
    if (cs == 8) return launch_cluster<R, 8, 1>(t, u, F, Y, norms, flag, st);
    if (cs == 4) return launch_cluster<R, 4, 1>(t, u, F, Y, norms, flag, st);
    if (cs == 2) return launch_cluster<R, 2, 1>(t, u, F, Y, norms, flag, st);
  }
  const int ppt = t.max_n <= 1024 ? 1 : (t.max_n <= 2048 ? 2 : 4);
  const int threads = (((t.max_n + ppt - 1) / ppt + 31) / 32) * 32;
  if (ppt == 1) return launch_ppt<R, 1, 1024>(t, threads, u, F, Y, norms, flag, st);
  if (ppt == 2) return launch_ppt<R, 2, 1024>(t, threads, u, F, Y, norms, flag, st);
  return launch_ppt<R, 4, 1024>(t, threads, u, F, Y, norms, flag, st);
}

// Packed launch: n_packs CTAs of gl1d_pack_threads<R>() threads, ppt slots per thread (map from the
// host packer).  A ring three steps deep (two ahead) unless that would not fit beside the exchange
// buffers: ppt = 4 keeps two (one ahead).  Every variant takes at most 196.7 KB of shared memory.
namespace {
template <typename R, int PPT>
struct PackCfg {
  static constexpr int nt = gl1d_pack_threads<R>();
  static constexpr int ring = PPT == 4 ? 2 : 3;
  static constexpr size_t smem = sizeof(cpx<R>) * (2 * ((size_t)nt * PPT + 2) + 2 * (size_t)ring * nt * PPT);
  static_assert(smem <= 232448, "packed GL1D kernel exceeds the shared memory of a CTA");
};
template <typename R, typename Fn>
cudaError_t with_pack_kernel(int ppt, Fn&& fn) {
  switch (ppt) {
    case 1: return fn(gl1d_pack_kernel<R, PackCfg<R, 1>::nt, 1, PackCfg<R, 1>::ring>, PackCfg<R, 1>::smem);
    case 2: return fn(gl1d_pack_kernel<R, PackCfg<R, 2>::nt, 2, PackCfg<R, 2>::ring>, PackCfg<R, 2>::smem);
    case 3: return fn(gl1d_pack_kernel<R, PackCfg<R, 3>::nt, 3, PackCfg<R, 3>::ring>, PackCfg<R, 3>::smem);
    case 4: return fn(gl1d_pack_kernel<R, PackCfg<R, 4>::nt, 4, PackCfg<R, 4>::ring>, PackCfg<R, 4>::smem);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

template <typename R>
cudaError_t gl1d_pack_occupancy(int ppt, int* ctas_per_sm) {
  return with_pack_kernel<R>(ppt, [&](auto kernel, size_t smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kernel, gl1d_pack_threads<R>(), smem);
  });
}

template <typename R>
cudaError_t launch_gl1d_pack(const Gl1dTile& t, const int32_t* map, int n_packs, int ppt, void* u, const void* F,
                             void* Y, int* flag, cudaStream_t st) {
  return with_pack_kernel<R>(ppt, [&](auto kernel, size_t smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<(unsigned)n_packs, gl1d_pack_threads<R>(), smem, st>>>(t, map, (cpx<R>*)u, (const cpx<R>*)F,
                                                                      (cpx<R>*)Y, flag);
    return cudaGetLastError();
  });
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
template cudaError_t gl1d_pack_occupancy<double>(int, int*);
template cudaError_t gl1d_pack_occupancy<float>(int, int*);
template cudaError_t launch_gl1d_apply<double>(const Gl1dTile&, const int32_t*, const void*, void*, cudaStream_t);
template cudaError_t launch_gl1d_apply<float>(const Gl1dTile&, const int32_t*, const void*, void*, cudaStream_t);

}  // namespace rsv
