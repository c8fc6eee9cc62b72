// Tensor-core (tcgen05) RK4 step of the dense propagator, FP32 mode.
//
//   u_{n+1} = u_n + D u_n + F_n      (D = RK4 step polynomial minus identity, see dense_kernels.cu)
//
// D u is computed as the real GEMM  [Dr; Di] (2n x n)  x  [Ur | Ui] (n x 2kg):
// rows 0..63 of a CTA's A tile are 64 rows of Re D, rows 64..127 the same rows
// of Im D, and  Re(Du) = DrUr - DiUi,  Im(Du) = DrUi + DiUr.  Operands are
// split into TF32 pairs (x = hi + lo, hi = tf32(x)) and three MMAs
// (hi*hi + hi*lo + lo*hi) give FP32-level products with FP32 accumulation in
// tensor memory.
//
// Grid: one cluster of CS = n/128 CTAs per block of 64 complex rows; CTA rank
// j of a cluster owns the K slice of 128 complex columns [128 j, 128 j + 128).
// Each CTA bulk-copies its pre-arranged A tile (hi, lo: 2 x 64 KB) and its X
// slice (hi, lo: 2 x 32 KB) into shared memory, issues 16 K-steps x 3 MMAs
// (M = 128, N = 64, K = 8) from one thread, reads the 128 x 64 partial from
// tensor memory and exchanges it through distributed shared memory: CTA j
// sums over the cluster the partials of its 64/CS complex rows (stacked rows
// r and 64 + r) and
// writes the new state, the snapshot, and the TF32 split of the new state
// in the operand layout of the next step.  All waits are bounded; a timeout
// sets the error flag.
#include <cuda_runtime.h>

#include <cstdlib>

#include "rsv_ops.h"
#include "tc_ptx.h"

namespace rsv {
namespace {

constexpr int kTileK = 128;                         // complex columns per K slice
constexpr int kTileRows = 64;                       // complex rows per cluster
constexpr int kM = 128, kN = 64;                    // MMA shape (real rows, 2 x 32 vector columns)
constexpr uint32_t kATileFloats = kM * kTileK;      // 16384 floats = 64 KB
constexpr uint32_t kXTileFloats = kN * kTileK;      // 8192 floats = 32 KB
constexpr uint32_t kSmemBytes = 4 * kATileFloats + 4 * kATileFloats + 4 * kXTileFloats + 4 * kXTileFloats + 64;
constexpr uint32_t kWaitTries = 1u << 24;
constexpr int kRedLd = kN + 1;

struct TcStepArgs {
  const float* A;     // [n/64][CS][2][kATileFloats]
  const float* Xin;   // [CS][2][kXTileFloats]
  float* Xout;
  const cpx<float>* uin;   // [kg][n]
  cpx<float>* uout;
  const cpx<float>* F;     // nullable
  cpx<float>* Y;           // nullable
  int n, kg, cs;
  int* err;
};

__global__ void __launch_bounds__(256, 1) dense_tc_step_kernel(TcStepArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* A_hi = reinterpret_cast<float*>(smem);
  float* A_lo = A_hi + kATileFloats;
  float* X_hi = A_lo + kATileFloats;
  float* X_lo = X_hi + kXTileFloats;
  uint64_t* bars = reinterpret_cast<uint64_t*>(X_lo + kXTileFloats);  // [0] loads, [1] mma
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + 2);
  float* red = A_hi;  // reused for the 128 x 64 partial once the MMAs have completed

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb = tc::cluster_id_x();
  const uint32_t j = tc::cluster_rank();
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tbase, 64);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tbase;

  if (tid == 0) {
    const float* at = a.A + ((size_t)mb * a.cs + j) * 2 * kATileFloats;
    const float* xt = a.Xin + (size_t)j * 2 * kXTileFloats;
    tc::mbar_arrive_expect_tx(&bars[0], 4 * (2 * kATileFloats + 2 * kXTileFloats));
    tc::bulk_g2s(A_hi, at, 4 * kATileFloats, &bars[0]);
    tc::bulk_g2s(A_lo, at + kATileFloats, 4 * kATileFloats, &bars[0]);
    tc::bulk_g2s(X_hi, xt, 4 * kXTileFloats, &bars[0]);
    tc::bulk_g2s(X_lo, xt + kXTileFloats, 4 * kXTileFloats, &bars[0]);
  }
  bool ok = tc::mbar_wait(&bars[0], 0, kWaitTries);
  if (tid == 0) {
    if (ok) {
      const uint32_t idesc = tc::idesc_tf32(kM, kN);
      const uint32_t lbo = 128, sbo_a = (kTileK / 4) * 128, sbo_x = (kTileK / 4) * 128;
#pragma unroll 1
      for (int ks = 0; ks < kTileK / 8; ++ks) {
        const uint64_t ah = tc::smem_desc(reinterpret_cast<char*>(A_hi) + ks * 256, lbo, sbo_a);
        const uint64_t al = tc::smem_desc(reinterpret_cast<char*>(A_lo) + ks * 256, lbo, sbo_a);
        const uint64_t xh = tc::smem_desc(reinterpret_cast<char*>(X_hi) + ks * 256, lbo, sbo_x);
        const uint64_t xl = tc::smem_desc(reinterpret_cast<char*>(X_lo) + ks * 256, lbo, sbo_x);
        tc::mma_tf32(tmem, ah, xh, idesc, ks > 0);
        tc::mma_tf32(tmem, ah, xl, idesc, true);
        tc::mma_tf32(tmem, al, xh, idesc, true);
      }
      tc::mma_commit(&bars[1]);
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bars[1])) : "memory");
    }
  }
  ok = tc::mbar_wait(&bars[1], 0, kWaitTries) && ok;
  tc::tc_fence_after();
  if (warp < 4) {
    const int row = 32 * warp + lane;
#pragma unroll
    for (int c = 0; c < kN; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) red[row * kRedLd + c + q] = ok ? v[q] : 0.f;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::cluster_sync();

  // cluster reduction + RK4 update: CTA j owns complex rows [rpc j, rpc j + rpc) of the
  // cluster's 64-row block (rpc = 64 / cs), i.e. stacked rows iloc and 64 + iloc
  {
    const int rpc = kTileRows / a.cs;
    for (int pidx = tid; pidx < rpc * 32; pidx += blockDim.x) {
      const int ii = pidx >> 5;
      const int v = pidx & 31;
      const int iloc = rpc * (int)j + ii;
      float pr = 0.f, pi = 0.f;
      {
        float rr[8], ri[8], ir[8], ix[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          if (p < a.cs) {
            rr[p] = tc::ld_peer_f32(tc::map_peer(&red[iloc * kRedLd + v], p));
            ri[p] = tc::ld_peer_f32(tc::map_peer(&red[iloc * kRedLd + 32 + v], p));
            ir[p] = tc::ld_peer_f32(tc::map_peer(&red[(64 + iloc) * kRedLd + v], p));
            ix[p] = tc::ld_peer_f32(tc::map_peer(&red[(64 + iloc) * kRedLd + 32 + v], p));
          }
        }
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          if (p < a.cs) {
            pr += rr[p] - ix[p];
            pi += ri[p] + ir[p];
          }
        }
      }
      const int i = (int)mb * kTileRows + iloc;
      if (v < a.kg && i < a.n) {
        const int64_t e = (int64_t)v * a.n + i;
        const cpx<float> u0 = a.uin[e];
        cpx<float> u1 = mk<float>(u0.re + pr, u0.im + pi);
        if (a.F) u1 = u1 + a.F[e];
        a.uout[e] = u1;
        if (a.Y) a.Y[e] = u0;
        const int js = i / kTileK, kk = i % kTileK;
        float* xo = a.Xout + (size_t)js * 2 * kXTileFloats;
        const float hr = tc::to_tf32(u1.re), hi = tc::to_tf32(u1.im);
        const uint32_t o_re = tc::kmajor_offset(v, kk, kTileK) / 4, o_im = tc::kmajor_offset(32 + v, kk, kTileK) / 4;
        xo[o_re] = hr;
        xo[kXTileFloats + o_re] = u1.re - hr;
        xo[o_im] = hi;
        xo[kXTileFloats + o_im] = u1.im - hi;
      }
    }
  }
  tc::cluster_sync();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
  if (!ok && tid == 0) atomicExch(a.err, 2);
}

// ---------------------------------------------------------------------------
// Persistent variant (no clusters): one launch marches a whole time tile with
// MB * CS CTAs, one per SM, all resident at once.  CTA (mb, j) keeps the A
// tile of row block mb and K slice j in shared memory for the whole tile.
//
// The test vectors are split into up to two independent chains of 16 vectors
// (32 real columns), each driven by its own four warps with its own operand
// buffer, mbarriers, tensor-memory columns and counters, so one chain's
// hand-off latency overlaps the other chain's work.  Per chain and step:
//   1. wait until row blocks 2j and 2j+1 have published the state (counter),
//      bulk-copy the TF32 hi / lo split of the state slice (32 KB);
//   2. two MMAs per K-step: A_hi x [X_hi | X_lo] (N = 64) and A_lo x X_hi
//      (N = 32), so the A tile is read from shared memory twice, not three times;
//   3. sum the three product groups out of tensor memory into the CTA's
//      128 x 32 partial, store it (L2) and count it in the row block's counter;
//   4. as owner of 64/CS rows of its row block, wait for all CS partials of the
//      step, bulk-copy its rows of them into shared memory (16 KB), sum them,
//      apply the RK4 update u <- u + D u + F (the owner keeps
//      its rows of u in registers for the whole tile), write the snapshot and
//      the hi / lo split of the new state, and count the publication.
// Partials, split states and counter targets are double-buffered by step
// parity: every row block reads every K slice, so no CTA runs more than one
// step ahead of any other within a chain.  Counters only grow (zeroed at the
// start of a march).  Spins are bounded in time and stop once any CTA has set
// the error flag.
// ---------------------------------------------------------------------------
constexpr int kChainVec = 16;                        // vectors per chain
constexpr int kChainN = 2 * kChainVec;               // real columns per chain (re, im)
constexpr int kMaxChains = 2;
constexpr uint32_t kXcFloats = 2 * kChainN * kTileK; // hi rows [0, 32) then lo rows [32, 64): 8192 floats
constexpr uint32_t kPartFloats = kM * kChainN;       // 128 x 32 partial of one CTA
constexpr uint32_t kGFloats = 2 * kTileRows * kChainN;   // the owner's rows of all CS partials: 16 KB
constexpr uint32_t kSmemPersistent = 4 * (2 * kATileFloats + kMaxChains * (kXcFloats + kGFloats)) + 256;
constexpr int kMarchThreads = 128 * kMaxChains;

struct TcMarchArgs {
  const float* A;
  float* X;                 // [chains][2][CS][kXcFloats]
  float* part;              // [chains][2][MB][CS][kPartFloats]
  int* cnt;                 // [chains][2][MB]  partials stored
  int* ready;               // [chains][MB]     owner publications
  cpx<float>* u;            // [2][kg][n]: state at n0 in slot n0 & 1, written back to slot (n0 + steps) & 1
  const cpx<float>* F;      // [steps][kg][n] or null
  cpx<float>* Y;            // [steps][kg][n] or null
  int64_t n0;
  int steps;
  int64_t n_forced;
  int y_first;
  int n, kg, cs, chains;
  int* err;
  uint64_t wait_ns;         // limit of each wait on another CTA's counter
  int stall;                // test hook: the first state wait of the tile targets a count nobody reaches
};

__device__ __forceinline__ void chain_bar(int chain) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + chain) : "memory");
}

__global__ void __launch_bounds__(kMarchThreads, 1) dense_tc_march_kernel(TcMarchArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* A_hi = reinterpret_cast<float*>(smem);
  float* A_lo = A_hi + kATileFloats;
  float* Xs = A_lo + kATileFloats;                                          // [chain][kXcFloats]
  float* Gs = Xs + kMaxChains * kXcFloats;                                  // [chain][kGFloats]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Gs + kMaxChains * kGFloats);  // [0] A, then 3 per chain
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + 1 + 3 * kMaxChains);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chain = warp >> 2;                  // warps 4c .. 4c + 3 drive chain c
  const int ctid = tid & 127;                   // thread index within the chain
  const int MB = a.n / kTileRows;
  const int mb = blockIdx.x / a.cs;
  const int j = blockIdx.x % a.cs;
  const volatile int* errv = a.err;
  if (tid == 0) {
    for (int b = 0; b < 1 + 3 * kMaxChains; ++b) tc::mbar_init(&bars[b], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tbase, 256);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tbase;
  if (tid == 0) {
    const float* at = a.A + ((size_t)mb * a.cs + j) * 2 * kATileFloats;
    tc::mbar_arrive_expect_tx(&bars[0], 4 * 2 * kATileFloats);
    tc::bulk_g2s(A_hi, at, 4 * kATileFloats, &bars[0]);
    tc::bulk_g2s(A_lo, at + kATileFloats, 4 * kATileFloats, &bars[0]);
  }
  bool ok = tc::mbar_wait(&bars[0], 0, 0xFFFFFFFFu);   // this CTA's own copy: never abandoned early
  __syncthreads();
  if (chain < a.chains) {
    float* X_sm = Xs + (size_t)chain * kXcFloats;
    uint64_t* bar_x = &bars[1 + 3 * chain];
    uint64_t* bar_m = &bars[2 + 3 * chain];
    uint64_t* bar_g = &bars[3 + 3 * chain];
    float* G_sm = Gs + (size_t)chain * kGFloats;   // [CS][re rows, im rows][rpc][kChainN]
    const uint32_t tcol = tmem + (uint32_t)(chain * 128);
    const size_t xset = (size_t)a.cs * kXcFloats;                // one parity
    float* Xg = a.X + (size_t)chain * 2 * xset;
    float* partg = a.part + (size_t)chain * 2 * MB * a.cs * kPartFloats;
    int* cnt = a.cnt + chain * 2 * MB;
    int* ready = a.ready + chain * MB;
    const int64_t rows = (int64_t)a.kg * a.n;
    const int v0 = chain * kChainVec;
    const uint32_t idesc_hx = tc::idesc_tf32(kM, 2 * kChainN);   // A_hi x [X_hi | X_lo]
    const uint32_t idesc_lx = tc::idesc_tf32(kM, kChainN);       // A_lo x X_hi
    const uint32_t sbo = (kTileK / 4) * 128;
    // owner pairs: rows [rpc j, rpc j + rpc) of the row block x 16 vectors, kPairs per thread
    const int rpc = kTileRows / a.cs;
    const int npairs = rpc * kChainVec;
    constexpr int kMaxPairs = kTileRows * kChainVec / 128;       // 8 (cs = 1)
    const int vl = ctid & 15;
    const int vg = v0 + vl;
    cpx<float> u_own[kMaxPairs];
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) {
      const int pidx = ctid + 128 * q;
      const int i = mb * kTileRows + rpc * j + (pidx >> 4);
      u_own[q] = (pidx < npairs && vg < a.kg) ? a.u[(size_t)(a.n0 & 1) * rows + (int64_t)vg * a.n + i]
                                               : mk<float>(0.f, 0.f);
    }
    // X slot layout: hi rows [0, 32) (re of 16 vectors, then im), lo rows [32, 64)
    auto write_x = [&](float* xo_par, int i, cpx<float> u1) {
      const int js = i / kTileK, kk = i % kTileK;
      float* xo = xo_par + (size_t)js * kXcFloats;
      const float hr = tc::to_tf32(u1.re), hi = tc::to_tf32(u1.im);
      __stcg(xo + tc::kmajor_offset(vl, kk, kTileK) / 4, hr);
      __stcg(xo + tc::kmajor_offset(kChainVec + vl, kk, kTileK) / 4, hi);
      __stcg(xo + tc::kmajor_offset(kChainN + vl, kk, kTileK) / 4, u1.re - hr);
      __stcg(xo + tc::kmajor_offset(kChainN + kChainVec + vl, kk, kTileK) / 4, u1.im - hi);
    };
    if (a.n0 == 0) {  // publish the initial state's split (later tiles find it from the previous tile)
#pragma unroll
      for (int q = 0; q < kMaxPairs; ++q) {
        const int pidx = ctid + 128 * q;
        if (pidx < npairs) write_x(Xg, mb * kTileRows + rpc * j + (pidx >> 4), u_own[q]);
      }
      chain_bar(chain);
      if (ctid == 0) tc::red_release_add(&ready[mb], 1);
    }
    // Every thread of the chain runs every step (named barriers need all 128);
    // after an error the waits return at once and the flag reports the failure.
    for (int s = 0; s < a.steps; ++s) {
      const int64_t n = a.n0 + s;
      const int par = (int)(n & 1);
      // forcing of this step for the owned pairs: loads in flight during the MMA phase
      const cpx<float>* Fs = (a.F != nullptr && n < a.n_forced) ? a.F + (size_t)s * rows : nullptr;
      cpx<float> fv[kMaxPairs];
#pragma unroll
      for (int q = 0; q < kMaxPairs; ++q) {
        const int pidx = ctid + 128 * q;
        const int i = mb * kTileRows + rpc * j + (pidx >> 4);
        fv[q] = (Fs != nullptr && pidx < npairs && vg < a.kg)
                    ? mk<float>(__ldcs(reinterpret_cast<const float*>(Fs + (int64_t)vg * a.n + i)),
                                __ldcs(reinterpret_cast<const float*>(Fs + (int64_t)vg * a.n + i) + 1))
                    : mk<float>(0.f, 0.f);
      }
      // 1. the state slice of this step
      if (ctid == 0) {
        const int target = a.cs * (int)(n + 1) + ((a.stall && s == 0) ? (1 << 30) : 0);
        const bool got = tc::spin_until_geq(&ready[2 * j], target, errv, a.wait_ns) &&
                         tc::spin_until_geq(&ready[2 * j + 1], target, errv, a.wait_ns);
        if (!got) {
          atomicExch(a.err, 2);
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar_x)) : "memory");
        } else {
          tc::fence_proxy_async_global();
          tc::mbar_arrive_expect_tx(bar_x, 4 * kXcFloats);
          tc::bulk_g2s(X_sm, Xg + (size_t)par * xset + (size_t)j * kXcFloats, 4 * kXcFloats, bar_x);
        }
      }
      // 2. products
      if (ctid == 0) {
        bool okx = tc::mbar_wait(bar_x, (uint32_t)(s & 1), 0xFFFFFFFFu) && *errv == 0;
        tc::tc_fence_after();
        if (okx) {
#pragma unroll 4
          for (int ks = 0; ks < kTileK / 8; ++ks) {
            const uint64_t ah = tc::smem_desc(reinterpret_cast<char*>(A_hi) + ks * 256, 128, sbo);
            const uint64_t al = tc::smem_desc(reinterpret_cast<char*>(A_lo) + ks * 256, 128, sbo);
            const uint64_t xx = tc::smem_desc(reinterpret_cast<char*>(X_sm) + ks * 256, 128, sbo);
            tc::mma_tf32(tcol, ah, xx, idesc_hx, ks > 0);
            tc::mma_tf32(tcol + 2 * kChainN, al, xx, idesc_lx, ks > 0);
          }
          tc::mma_commit(bar_m);
        } else {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar_m)) : "memory");
        }
      }
      ok = tc::mbar_wait(bar_m, (uint32_t)(s & 1), 0xFFFFFFFFu) && ok && *errv == 0;
      tc::tc_fence_after();
      // 3. partial: hi*hi + hi*lo + lo*hi, one row per thread
      float* pb = partg + (((size_t)par * MB + mb) * a.cs + j) * kPartFloats;
      {
        const int qw = warp & 3;
        const int row = 32 * qw + lane;
        const uint32_t tl = tcol + ((uint32_t)(32 * qw) << 16);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float x0[16], x1[16], x2[16];
          tc::tmem_ld16(tl + 16 * h, x0);
          tc::tmem_ld16(tl + kChainN + 16 * h, x1);
          tc::tmem_ld16(tl + 2 * kChainN + 16 * h, x2);
          float4* dst = reinterpret_cast<float4*>(pb + row * kChainN + 16 * h);
#pragma unroll
          for (int c = 0; c < 4; ++c)
            __stcg(dst + c, make_float4(x0[4 * c] + x1[4 * c] + x2[4 * c], x0[4 * c + 1] + x1[4 * c + 1] + x2[4 * c + 1],
                                        x0[4 * c + 2] + x1[4 * c + 2] + x2[4 * c + 2],
                                        x0[4 * c + 3] + x1[4 * c + 3] + x2[4 * c + 3]));
        }
      }
      tc::tc_fence_before();
      chain_bar(chain);
      if (ctid == 0) tc::red_release_add(&cnt[par * MB + mb], 1);
      // 4. owner: all partials of the row block for this step; the owner's rows of every
      //    partial (rpc real-part rows and rpc imaginary-part rows) come in by bulk copies
      const float* pbase = partg + ((size_t)par * MB + mb) * a.cs * kPartFloats;
      if (ctid == 0) {
        if (!tc::spin_until_geq(&cnt[par * MB + mb], a.cs * (int)((n >> 1) + 1), errv, a.wait_ns)) {
          atomicExch(a.err, 2);
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar_g)) : "memory");
        } else {
          tc::fence_proxy_async_global();
          const uint32_t rows_bytes = (uint32_t)rpc * kChainN * 4;
          tc::mbar_arrive_expect_tx(bar_g, 2u * (uint32_t)a.cs * rows_bytes);
          for (int p = 0; p < a.cs; ++p) {
            const float* src = pbase + (size_t)p * kPartFloats;
            float* dst = G_sm + (size_t)p * 2 * rpc * kChainN;
            tc::bulk_g2s(dst, src + (size_t)(rpc * j) * kChainN, rows_bytes, bar_g);
            tc::bulk_g2s(dst + rpc * kChainN, src + (size_t)(64 + rpc * j) * kChainN, rows_bytes, bar_g);
          }
        }
      }
      if (!tc::mbar_wait(bar_g, (uint32_t)(s & 1), 0xFFFFFFFFu)) atomicExch(a.err, 2);
      cpx<float>* Ys = (a.Y != nullptr && s >= a.y_first) ? a.Y + (size_t)s * rows : nullptr;
      float* xo_par = Xg + (size_t)(1 - par) * xset;
#pragma unroll
      for (int q = 0; q < kMaxPairs; ++q) {
        const int pidx = ctid + 128 * q;
        if (pidx < npairs) {
          const int il = pidx >> 4;
          const int iloc = rpc * j + il;
          float prr = 0.f, pri = 0.f, pir = 0.f, pii = 0.f;
          float t0[8], t1[8], t2[8], t3[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            if (p < a.cs) {
              const float* gr = G_sm + (size_t)p * 2 * rpc * kChainN + il * kChainN;
              const float* gi = gr + rpc * kChainN;
              t0[p] = gr[vl];
              t1[p] = gr[kChainVec + vl];
              t2[p] = gi[vl];
              t3[p] = gi[kChainVec + vl];
            }
          }
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            if (p < a.cs) {
              prr += t0[p];
              pri += t1[p];
              pir += t2[p];
              pii += t3[p];
            }
          }
          const int i = mb * kTileRows + iloc;
          const cpx<float> u0 = u_own[q];
          cpx<float> u1 = mk<float>(u0.re + (prr - pii) + fv[q].re, u0.im + (pri + pir) + fv[q].im);
          if (vg >= a.kg) u1 = mk<float>(0.f, 0.f);
          if (Ys != nullptr && vg < a.kg) __stcs(reinterpret_cast<float2*>(Ys + (int64_t)vg * a.n + i), make_float2(u0.re, u0.im));
          write_x(xo_par, i, u1);
          u_own[q] = u1;
        }
      }
      chain_bar(chain);
      if (ctid == 0) tc::red_release_add(&ready[mb], 1);
    }
    // state at the end of the tile
    const int64_t nend = a.n0 + a.steps;
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) {
      const int pidx = ctid + 128 * q;
      const int i = mb * kTileRows + rpc * j + (pidx >> 4);
      if (pidx < npairs && vg < a.kg) a.u[(size_t)(nend & 1) * rows + (int64_t)vg * a.n + i] = u_own[q];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
  if (!ok && (tid & 127) == 0) atomicExch(a.err, 2);
}

// A tiles from the FP64 matrix (conj-transposed for the adjoint): tile (mb, j) rows
// r < 64: Re M[64 mb + r][128 j + k], r >= 64: Im M[64 mb + r - 64][128 j + k]; hi/lo TF32 split.
__global__ void arrange_a_kernel(int n, int cs, const cpx<double>* __restrict__ M, bool conj_t, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over (mb, j, r, k)
  const int64_t total = (int64_t)(n / kTileRows) * cs * kM * kTileK;
  if (e >= total) return;
  const int k = (int)(e % kTileK);
  const int r = (int)((e / kTileK) % kM);
  const int j = (int)((e / ((int64_t)kTileK * kM)) % cs);
  const int mb = (int)(e / ((int64_t)kTileK * kM * cs));
  const int row = mb * kTileRows + (r & 63), col = j * kTileK + k;
  const cpx<double> m = conj_t ? conjg(M[(int64_t)col * n + row]) : M[(int64_t)row * n + col];
  const double x = (r < 64) ? m.re : m.im;
  const float hi = tc::to_tf32((float)x);
  const float lo = (float)(x - (double)hi);
  float* tile = out + ((size_t)mb * cs + j) * 2 * kATileFloats;
  const uint32_t o = tc::kmajor_offset(r, k, kTileK) / 4;
  tile[o] = hi;
  tile[kATileFloats + o] = lo;
}

}  // namespace

// Shapes of the tensor-core kernels: n a multiple of 128 with CS = n / 128 K slices, and
// CS dividing the 64 rows of a row block (each of the CS CTAs of a row block owns
// 64 / CS of its rows): CS in {1, 2, 4, 8}, n in {128, 256, 512, 1024}.  Other n take
// the CUDA-core step.
static bool tc_shape_ok(int n) {
  if (n % kTileK != 0) return false;
  const int cs = n / kTileK;
  return cs >= 1 && cs <= 8 && kTileRows % cs == 0;
}

bool dense_tc_supported(rsv_operator op, int kg) {
  if (op->prec != RSV_PREC_FP32 || op->kind != RSV_OP_DENSE) return false;
  if (op->tc_disabled) return false;
  if (!tc_shape_ok((int)op->n) || kg > 32) return false;
  return op->tc_tiles[0] != nullptr;
}

size_t dense_tc_scratch_bytes(rsv_operator op) {
  return (size_t)2 * (op->n / kTileK) * 2 * kXTileFloats * sizeof(float);
}

// Build the hi/lo A tiles of D and D^H (after the FP64 propagator build).
rsv_status dense_tc_prepare(rsv_operator op, const void* d64_direct) {
  const int n = (int)op->n;
  if (op->prec != RSV_PREC_FP32 || !tc_shape_ok(n) || op->tc_disabled) return RSV_OK;
  const int cs = n / kTileK;
  const size_t floats = (size_t)(n / kTileRows) * cs * 2 * kATileFloats;
  for (int d = 0; d < 2; ++d) {
    if (!op->tc_tiles[d]) {
      cudaError_t e = cudaMalloc(&op->tc_tiles[d], floats * sizeof(float));
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core tiles");
      op->dev.push_back(op->tc_tiles[d]);
    }
    const int64_t total = (int64_t)(n / kTileRows) * cs * kM * kTileK;
    arrange_a_kernel<<<(unsigned)((total + 255) / 256), 256, 0, op->stream>>>(
        n, cs, (const cpx<double>*)d64_direct, d == 1, (float*)op->tc_tiles[d]);
  }
  cudaError_t e = cudaFuncSetAttribute(dense_tc_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_tc_march_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemPersistent);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core tiles");
  // The persistent tile kernel needs all of its CTAs resident at once (one per SM).
  op->tc_persistent = false;
  const int MB = n / kTileRows;
  if (!op->d_ready) {
    e = cudaMalloc(&op->d_ready, sizeof(int) * kMaxChains * 3 * MB);
    if (e == cudaSuccess) op->dev.push_back(op->d_ready);
    if (e == cudaSuccess) e = cudaMalloc(&op->tc_acc, sizeof(float) * kMaxChains * 2 * MB * cs * kPartFloats);
    if (e == cudaSuccess) op->dev.push_back(op->tc_acc);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core march buffers");
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_tc_march_kernel, kMarchThreads, kSmemPersistent);
  if (e != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  op->tc_max_clusters = per_sm * op->sm_count;  // resident CTAs
  const char* env = getenv("RSV_DENSE_PERSISTENT");
  op->tc_persistent = per_sm * op->sm_count >= MB * cs && !(env != nullptr && env[0] == '0');
  return RSV_OK;
}

// Operand buffers of the persistent kernel (per chain, two step parities).
size_t dense_tc_chain_x_bytes(rsv_operator op) {
  return (size_t)kMaxChains * 2 * (op->n / kTileK) * kXcFloats * sizeof(float);
}

// A whole tile of steps in one persistent launch (requires op->tc_persistent).
cudaError_t dense_tc_march_tile(rsv_operator op, int kg, bool adjoint, int64_t n0, int steps, int64_t n_forced,
                                int y_first, void* state, const void* F, void* Y, void* xbuf) {
  const int n = (int)op->n;
  const int cs = n / kTileK;
  const int MB = n / kTileRows;
  TcMarchArgs a;
  a.A = (const float*)op->tc_tiles[adjoint ? 1 : 0];
  a.X = (float*)xbuf;
  a.part = (float*)op->tc_acc;
  a.cnt = (int*)op->d_ready;                       // [chains][2][MB]
  a.ready = (int*)op->d_ready + kMaxChains * 2 * MB;  // [chains][MB]
  a.u = (cpx<float>*)state;
  a.F = (const cpx<float>*)F;
  a.Y = (cpx<float>*)Y;
  a.n0 = n0;
  a.steps = steps;
  a.n_forced = n_forced;
  a.y_first = y_first;
  a.n = n;
  a.kg = kg;
  a.cs = cs;
  a.chains = (kg + kChainVec - 1) / kChainVec;
  a.err = op->d_flag;
  a.wait_ns = op->wait_limit_ns;
  a.stall = op->test_stall_wait ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (n0 == 0) {
    e = cudaMemsetAsync(op->d_ready, 0, sizeof(int) * kMaxChains * 3 * MB, op->stream);
  }
  if (e != cudaSuccess) return e;
  dense_tc_march_kernel<<<MB * cs, kMarchThreads, kSmemPersistent, op->stream>>>(a);
  return cudaGetLastError();
}

// One step; xbuf holds two X operand sets (ping-pong by step parity).
cudaError_t dense_tc_step(rsv_operator op, int kg, bool adjoint, int64_t step, const void* uin, void* uout,
                          const void* F, void* Y, void* xbuf) {
  const int n = (int)op->n;
  const int cs = n / kTileK;
  const size_t xset = (size_t)cs * 2 * kXTileFloats;
  TcStepArgs a;
  a.A = (const float*)op->tc_tiles[adjoint ? 1 : 0];
  a.Xin = (const float*)xbuf + (size_t)(step & 1) * xset;
  a.Xout = (float*)xbuf + (size_t)((step + 1) & 1) * xset;
  a.uin = (const cpx<float>*)uin;
  a.uout = (cpx<float>*)uout;
  a.F = (const cpx<float>*)F;
  a.Y = (cpx<float>*)Y;
  a.n = n;
  a.kg = kg;
  a.cs = cs;
  a.err = op->d_flag;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((n / kTileRows) * cs), 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = op->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, dense_tc_step_kernel, a);
}

}  // namespace rsv
