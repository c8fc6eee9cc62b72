// Forcing synthesis and DFT analysis on the tensor cores (FP32 mode).
//
// Both contractions of a time tile are real GEMMs after expanding complex
// numbers into (re, im) pairs:
//   synthesis  F[tau][r]     = sum_j W[tau][j] C[j][r]          (Sec. 2.3, Eq. forceFseries)
//   analysis   acc[j][r]    += sum_s conj(W[s][j]) Y[s][r]       (Sec. 2.1, Eq. fourier)
// with W the exact twiddles of the tile.  The M dimension is the long one
// (state rows r, 128 per CTA), N the output columns (stage times or
// frequencies, re/im expanded, <= 512, accumulated in tensor memory), and K
// the contracted one (frequencies or tile steps, re/im expanded).
//
// The twiddle operand B (N x K) is the same for every CTA: one small kernel
// builds it per tile in global memory, already TF32 hi/lo split and in the
// K-major no-swizzle operand layout, 16 K-columns per chunk.  Each CTA streams
// K in chunks of 16 through two shared-memory stages: threads read its 128
// rows of the long operand (coalesced along r), split them into TF32 hi/lo
// and store them K-major; one thread bulk-copies the B chunk and issues the
// MMAs (3 per K-step: hi*hi, hi*lo, lo*hi).  The epilogue reads tensor memory
// (one row per thread) and writes F, or adds the tile's sums into the FP64
// accumulators.  Waits are bounded; a timeout sets the error flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "rsv_ops.h"
#include "tc_ptx.h"

namespace rsv {
namespace {

constexpr int kRowsCta = 128;
constexpr int kKc = 16;                              // K columns per chunk
constexpr int kMaxN = 512;
constexpr uint32_t kAStageFloats = kRowsCta * kKc;   // per hi / lo
constexpr uint32_t kBStageFloats = kMaxN * kKc;      // per hi / lo (N padded to 512)
constexpr uint32_t kSmem = 4 * 2 * (2 * kAStageFloats + 2 * kBStageFloats) + 128;
constexpr uint32_t kTries = 1u << 24;

enum Mode { SYNTH_C = 0, SYNTH_R = 1, ANAL_C = 2, ANAL_R = 3 };

struct ContractArgs {
  int mode;
  int64_t rows;
  int N;                   // output columns (multiple of 16, <= 512)
  int K;                   // contracted columns (multiple of 16)
  int n_tau;               // synthesis: stage times in this call
  int tau0;                // synthesis: first stage time of this call
  int n_omega;
  const void* src;         // coefficients [n_omega][coef_stride] or snapshots [steps][rows]
  int64_t src_stride;
  int s0, s1;              // analysis: valid tile steps [s0, s1)
  const float* B;          // [K / 16][2][kMaxN x 16] pre-split twiddle chunks
  void* out;               // synthesis: F [n_tau][rows]; analysis: acc (cpx<double>) [n_omega][acc_stride]
  int64_t acc_stride;
  int* err;
};

// The long operand of one K chunk as this thread's share, loaded into registers:
// complex modes: 4 (re, im) pairs = 4 rows x one contracted pair index each;
// real analysis: 8 values.  Zero outside the valid range.
struct AShare {
  float v[8];
};

__device__ __forceinline__ void load_share(const ContractArgs& a, int64_t r0, int kc, int tid, AShare& sh) {
  if (a.mode == ANAL_R) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      const int kk = e >> 7, rr = e & 127;
      const int s = kc * kKc + kk;
      const int64_t r = r0 + rr;
      sh.v[q] = (r < a.rows && s >= a.s0 && s < a.s1) ? __ldg(reinterpret_cast<const float*>(a.src) + (int64_t)s * a.rows + r)
                                                        : 0.f;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q;
    const int jj = e >> 7, rr = e & 127;
    const int idx = kc * (kKc / 2) + jj;  // frequency (synthesis) or tile step (analysis)
    const int64_t r = r0 + rr;
    bool valid = r < a.rows;
    int64_t off;
    if (a.mode == ANAL_C) {
      valid = valid && idx >= a.s0 && idx < a.s1;
      off = (int64_t)idx * a.rows + r;
    } else {
      valid = valid && idx < a.n_omega;
      off = (int64_t)idx * a.src_stride + r;
    }
    const float2 c = valid ? __ldg(reinterpret_cast<const float2*>(a.src) + off) : make_float2(0.f, 0.f);
    sh.v[2 * q] = c.x;
    sh.v[2 * q + 1] = c.y;
  }
}

__device__ __forceinline__ void store_share(const ContractArgs& a, int tid, const AShare& sh, float* A_hi, float* A_lo) {
  if (a.mode == ANAL_R) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      const int kk = e >> 7, rr = e & 127;
      const float hi = tc::to_tf32(sh.v[q]);
      const uint32_t o = tc::kmajor_offset(rr, kk, kKc) / 4;
      A_hi[o] = hi;
      A_lo[o] = sh.v[q] - hi;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q;
    const int jj = e >> 7, rr = e & 127;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const float x = sh.v[2 * q + part];
      const float hi = tc::to_tf32(x);
      const uint32_t o = tc::kmajor_offset(rr, 2 * jj + part, kKc) / 4;
      A_hi[o] = hi;
      A_lo[o] = x - hi;
    }
  }
}

__global__ void __launch_bounds__(256, 1) tc_contract_kernel(ContractArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* sA = reinterpret_cast<float*>(smem);                    // [2 stages][hi, lo][kAStageFloats]
  float* sB = sA + 2 * 2 * kAStageFloats;                        // [2 stages][hi, lo][kBStageFloats]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * 2 * kBStageFloats);  // [0,1] B loaded, [2,3] MMA done
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsCta;
  if (tid == 0) {
    for (int b = 0; b < 4; ++b) tc::mbar_init(&bars[b], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tbase, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tbase;
  const int chunks = a.K / kKc;
  const uint32_t sbo_a = (kKc / 4) * 128, sbo_b = (kKc / 4) * 128;
  const uint32_t bchunk_bytes = 4u * (uint32_t)a.N * kKc;  // one of hi / lo, only the N used rows
  bool ok = true;
  uint32_t mma_phase[2] = {0, 0};
  uint32_t load_phase[2] = {0, 0};
  AShare nxt;
  load_share(a, r0, 0, tid, nxt);
  for (int kc = 0; kc < chunks; ++kc) {
    const int st = kc & 1;
    float* A_hi = sA + st * 2 * kAStageFloats;
    float* A_lo = A_hi + kAStageFloats;
    float* B_hi = sB + st * 2 * kBStageFloats;
    float* B_lo = B_hi + kBStageFloats;
    const AShare cur = nxt;
    if (kc + 1 < chunks) load_share(a, r0, kc + 1, tid, nxt);  // in flight during this chunk
    if (kc >= 2) {  // the MMAs of chunk kc - 2 read this stage
      ok = tc::mbar_wait(&bars[2 + st], mma_phase[st], kTries) && ok;
      mma_phase[st] ^= 1;
    }
    if (tid == 0) {
      const float* bsrc = a.B + (size_t)kc * 2 * kBStageFloats;
      tc::mbar_arrive_expect_tx(&bars[st], 2 * bchunk_bytes);
      tc::bulk_g2s(B_hi, bsrc, bchunk_bytes, &bars[st]);
      tc::bulk_g2s(B_lo, bsrc + kBStageFloats, bchunk_bytes, &bars[st]);
    }
    store_share(a, tid, cur, A_hi, A_lo);
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      ok = tc::mbar_wait(&bars[st], load_phase[st], kTries) && ok;
      tc::tc_fence_after();
      if (ok) {
        for (int ks = 0; ks < kKc / 8; ++ks) {
          const uint64_t ah = tc::smem_desc(reinterpret_cast<char*>(A_hi) + ks * 256, 128, sbo_a);
          const uint64_t al = tc::smem_desc(reinterpret_cast<char*>(A_lo) + ks * 256, 128, sbo_a);
          for (int nh = 0; nh < a.N; nh += 256) {
            const int nn = min(256, a.N - nh);
            const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)nn);
            const uint64_t bh = tc::smem_desc(reinterpret_cast<char*>(B_hi) + ks * 256 + (nh / 8) * sbo_b, 128, sbo_b);
            const uint64_t bl = tc::smem_desc(reinterpret_cast<char*>(B_lo) + ks * 256 + (nh / 8) * sbo_b, 128, sbo_b);
            const uint32_t d = tmem + (uint32_t)nh;
            tc::mma_tf32(d, ah, bh, idesc, kc > 0 || ks > 0);
            tc::mma_tf32(d, ah, bl, idesc, true);
            tc::mma_tf32(d, al, bh, idesc, true);
          }
        }
        tc::mma_commit(&bars[2 + st]);
      } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bars[2 + st])) : "memory");
      }
    }
    load_phase[st] ^= 1;
  }
  // wait for the last chunks' MMAs
  for (int st = 0; st < 2; ++st) {
    const int issued = chunks > st ? (chunks - 1 - st) / 2 + 1 : 0;   // commits on this stage
    const int waited = chunks > st + 2 ? (chunks - 1 - st) / 2 : 0;   // waits done in the loop
    if (issued > waited) ok = tc::mbar_wait(&bars[2 + st], mma_phase[st], kTries) && ok;
  }
  tc::tc_fence_after();
  // epilogue: warps 0-3 own TMEM lanes (rows) 0-127
  if (warp < 4) {
    const int64_t r = r0 + 32 * warp + lane;
    for (int c = 0; c < a.N; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
      if (!ok || r >= a.rows) continue;
      if (a.mode == SYNTH_C) {
        cpx<float>* F = reinterpret_cast<cpx<float>*>(a.out);
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const int tau = (c + q) >> 1;
          if (tau < a.n_tau) F[(int64_t)(a.tau0 + tau) * a.rows + r] = mk<float>(v[q], v[q + 1]);
        }
      } else if (a.mode == SYNTH_R) {
        float* F = reinterpret_cast<float*>(a.out);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int tau = c + q;
          if (tau < a.n_tau) F[(int64_t)(a.tau0 + tau) * a.rows + r] = v[q];
        }
      } else {
        // 8 complex accumulators per TMEM load: issue the 8 FP64 reads before any add / write
        cpx<double>* __restrict__ acc = reinterpret_cast<cpx<double>*>(a.out);
        double2 old[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = (c >> 1) + q;
          old[q] = j < a.n_omega ? __ldcg(reinterpret_cast<const double2*>(acc + (int64_t)j * a.acc_stride + r))
                                 : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = (c >> 1) + q;
          if (j < a.n_omega)
            __stcg(reinterpret_cast<double2*>(acc + (int64_t)j * a.acc_stride + r),
                   make_double2(old[q].x + (double)v[2 * q], old[q].y + (double)v[2 * q + 1]));
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
  if (!ok && tid == 0) atomicExch(a.err, 2);
}

// B operand of the tile: element (nrow, k) in chunk k / 16, TF32 hi / lo, K-major.
__global__ void build_b_kernel(ContractArgs a, TileGeom g, const cpx<float>* __restrict__ tw,
                               const int64_t* __restrict__ pj, const float* __restrict__ cw, float* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)kMaxN * a.K) return;
  const int nrow = (int)(e / a.K), k = (int)(e % a.K);
  float val = 0.f;
  if (nrow < a.N) {
    switch (a.mode) {
      case SYNTH_C: {
        const int tau = nrow >> 1, q = nrow & 1, j = k >> 1, part = k & 1;
        if (tau < a.n_tau && j < a.n_omega) {
          const cpx<float> w = tw[phase_index(g.sgn * pj[j], 2 * g.n0 + (int64_t)(a.tau0 + tau) * g.tau_stride, g.m4)];
          // Fr = sum (Tr Cr - Ti Ci), Fi = sum (Ti Cr + Tr Ci)
          val = q == 0 ? (part == 0 ? w.re : -w.im) : (part == 0 ? w.im : w.re);
        }
        break;
      }
      case SYNTH_R: {
        const int tau = nrow, j = k >> 1, part = k & 1;
        if (tau < a.n_tau && j < a.n_omega) {
          const cpx<float> w = tw[phase_index(g.sgn * pj[j], 2 * g.n0 + (int64_t)(a.tau0 + tau) * g.tau_stride, g.m4)];
          val = cw[j] * (part == 0 ? w.re : -w.im);
        }
        break;
      }
      case ANAL_C: {
        const int j = nrow >> 1, q = nrow & 1, s = k >> 1, part = k & 1;
        if (j < a.n_omega && s >= a.s0 && s < a.s1) {
          const cpx<float> w = tw[phase_index(g.sgn * pj[j], 2 * (g.n0 + s), g.m4)];
          // conj(w) y: re = Tr yr + Ti yi, im = Tr yi - Ti yr
          val = q == 0 ? (part == 0 ? w.re : w.im) : (part == 0 ? -w.im : w.re);
        }
        break;
      }
      default: {
        const int j = nrow >> 1, q = nrow & 1, s = k;
        if (j < a.n_omega && s >= a.s0 && s < a.s1) {
          const cpx<float> w = tw[phase_index(g.sgn * pj[j], 2 * (g.n0 + s), g.m4)];
          val = q == 0 ? w.re : -w.im;
        }
      }
    }
  }
  const float hi = tc::to_tf32(val);
  const int kc = k / kKc, kk = k % kKc;
  float* chunk = B + (size_t)kc * 2 * kBStageFloats;
  const uint32_t o = tc::kmajor_offset(nrow, kk, kKc) / 4;
  chunk[o] = hi;
  chunk[kBStageFloats + o] = val - hi;
}

int round16(int x) { return (x + 15) / 16 * 16; }

cudaError_t run(ContractArgs& a, const TileGeom& g, rsv_operator op) {
  const size_t bbytes = (size_t)(a.K / kKc) * 2 * kBStageFloats * sizeof(float);
  if (ensure(op->ws_tcb, bbytes) != RSV_OK) return cudaErrorMemoryAllocation;
  a.B = (const float*)op->ws_tcb.ptr;
  a.err = op->d_flag;
  const int64_t total = (int64_t)kMaxN * a.K;
  build_b_kernel<<<(unsigned)((total + 255) / 256), 256, 0, op->stream>>>(a, g, (const cpx<float>*)op->d_tw, op->d_pj,
                                                                          op->d_cw, (float*)op->ws_tcb.ptr);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(tc_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    attr_set = true;
  }
  const unsigned blocks = (unsigned)((a.rows + kRowsCta - 1) / kRowsCta);
  tc_contract_kernel<<<blocks, 256, kSmem, op->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool tc_contract_supported(rsv_operator op, bool synth) {
  if (op->prec != RSV_PREC_FP32 || op->tc_contract_disabled) return false;
  return synth || round16(2 * op->n_omega) <= kMaxN;
}

// Stage times are processed in calls of at most 512 output columns (256 complex).
cudaError_t tc_synth(rsv_operator op, const TileGeom& g, const void* fhat, void* F) {
  const int total = g.n_tau > 0 ? g.n_tau : 2 * g.steps + 1;
  const int per_call = op->real_state ? kMaxN : kMaxN / 2;
  cudaError_t e = cudaSuccess;
  for (int t0 = 0; t0 < total && e == cudaSuccess; t0 += per_call) {
    ContractArgs a = {};
    a.mode = op->real_state ? SYNTH_R : SYNTH_C;
    a.rows = g.rows;
    a.tau0 = t0;
    a.n_tau = std::min(per_call, total - t0);
    a.n_omega = g.n_omega;
    a.N = op->real_state ? round16(a.n_tau) : round16(2 * a.n_tau);
    a.K = round16(2 * g.n_omega);
    a.src = fhat;
    a.src_stride = g.coef_stride;
    a.out = F;
    e = run(a, g, op);
  }
  return e;
}

cudaError_t tc_analysis(rsv_operator op, const TileGeom& g, const void* Y, int s0, int s1, cpx<double>* acc,
                        int64_t acc_stride) {
  ContractArgs a = {};
  a.mode = op->real_state ? ANAL_R : ANAL_C;
  a.rows = g.rows;
  a.n_omega = g.n_omega;
  a.N = round16(2 * g.n_omega);
  a.K = op->real_state ? round16(g.steps) : round16(2 * g.steps);
  a.s0 = s0;
  a.s1 = s1;
  a.src = Y;
  a.out = acc;
  a.acc_stride = acc_stride;
  return run(a, g, op);
}

}  // namespace rsv
