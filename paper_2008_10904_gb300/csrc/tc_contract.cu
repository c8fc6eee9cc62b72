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

// ---------------------------------------------------------------------------
// Pipelined persistent variant (long operand streamed by bulk copies).
//
// One CTA per SM walks the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// with warp roles connected by mbarrier rings:
//   warp 12 (one thread) producer: bulk-copies each K chunk of the long operand
//                        in its storage precision into a 4-deep raw ring;
//   warp 14 (one thread) producer: bulk-copies the chunk's pre-split twiddles
//                        into a 2-deep B ring;
//   warps 0-3            converters: one row each, raw value -> TF32 hi / lo in
//                        the K-major operand layout (2 stages);
//   warp 13 (one thread) MMA issuer: 3 TF32 MMAs per K-step and N half into the
//                        tile's tensor-memory accumulator, commits release the
//                        operand stages and, after the last chunk, the tile;
//   warps 4-11           epilogue: two warps per tensor-memory lane quadrant,
//                        each taking half of the columns, 32 columns per load;
//                        tensor memory -> F, or += FP64 accumulators; then
//                        release the accumulator for the next tile.
// The chunk sequence runs on across tiles, so the next tile's operands stream
// in during the current tile's epilogue.  Every wait is bounded and also
// returns once another role has aborted; on abort the producer and the MMA
// issuer drain what they issued (bounded) before the CTA frees tensor memory.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int round16c(int x) { return (x + 15) / 16 * 16; }

// Ring depths: the twiddle operand of every sub-tile streams from L2 (about 512 KB per row tile), so
// its ring is four chunks deep; a slot holds one sub-tile's 256 rows (hi and lo), half of a global
// chunk.  The raw long-operand ring is eight chunks deep.  Total 224.25 KB of shared memory.
constexpr int kRawRing = 8;
constexpr int kAStages = 2;
constexpr int kBRing = 4;
constexpr uint32_t kBRingFloats = 256 * kKc;          // per hi / lo: one sub-tile's rows
constexpr uint32_t kRawBytes = kRowsCta * kKc * 4;   // 128 rows x 16 real K values
constexpr int kPipeThreads = 480;                    // 15 warps, roles below

struct PipeBars {
  uint64_t raw_full[kRawRing], raw_empty[kRawRing];
  uint64_t a_full[kAStages], a_empty[kAStages];
  uint64_t b_full[kBRing], b_empty[kBRing];
  uint64_t acc_full[2], acc_empty[2];   // two tensor-memory accumulators of 256 columns
  int abort_flag;
};

// the barriers sit behind the operand rings; their reserve is sizeof(PipeBars) rounded up
constexpr uint32_t kPipeBarBytes = (uint32_t)((sizeof(PipeBars) + 127) / 128 * 128);
constexpr uint32_t kPipeSmem =
    kRawRing * kRawBytes + kAStages * 2 * kAStageFloats * 4 + kBRing * 2 * kBRingFloats * 4 + kPipeBarBytes;
// dynamic shared memory plus up to 1 KB for the static variable and the 1024-byte alignment
static_assert(kPipeSmem + 1024 <= 232448, "pipelined contraction exceeds the shared memory of a CTA");

__device__ __forceinline__ bool pwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return tc::mbar_wait(bar, parity, 0xFFFFFFFFu, abort_flag);
}

__device__ __forceinline__ void pabort(PipeBars* pb, int* err) {
  *reinterpret_cast<volatile int*>(&pb->abort_flag) = 1;
  atomicExch(err, 2);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Raw layout of one chunk in shared memory: complex modes [8][128] float2
// (pair index jj = frequency or step within the chunk), real analysis
// [16][128] float.  Only the valid pair indices and rows are copied.
__device__ __forceinline__ uint32_t issue_raw(const ContractArgs& a, int64_t r0, int nr, int kc, unsigned char* raw,
                                              uint64_t* bar) {
  const bool real = a.mode == ANAL_R;
  const int npair = real ? kKc : kKc / 2;
  const uint32_t esz = real ? 4 : 8;
  int lo = kc * npair, hi = lo + npair;
  if (a.mode == ANAL_C || a.mode == ANAL_R) {
    lo = max(lo, a.s0);
    hi = min(hi, a.s1);
  } else {
    hi = min(hi, a.n_omega);
  }
  const uint32_t bytes_row = (uint32_t)nr * esz;
  const uint32_t total = hi > lo ? (uint32_t)(hi - lo) * bytes_row : 0u;
  tc::mbar_arrive_expect_tx(bar, total);
  const int64_t stride = (a.mode == ANAL_C || a.mode == ANAL_R) ? a.rows : a.src_stride;
  for (int idx = lo; idx < hi; ++idx) {
    const unsigned char* src = reinterpret_cast<const unsigned char*>(a.src) + ((int64_t)idx * stride + r0) * esz;
    tc::bulk_g2s(raw + (uint32_t)(idx - kc * npair) * kRowsCta * esz, src, bytes_row, bar);
  }
  return total;
}

__device__ __forceinline__ void convert_row(const ContractArgs& a, int64_t r0, int kc, int rr, const unsigned char* raw,
                                            float* A_hi, float* A_lo) {
  const bool row_ok = r0 + rr < a.rows;
  float x[kKc];
  if (a.mode == ANAL_R) {
    const float* rv = reinterpret_cast<const float*>(raw);
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      const int s = kc * kKc + kk;
      x[kk] = (row_ok && s >= a.s0 && s < a.s1) ? rv[kk * kRowsCta + rr] : 0.f;
    }
  } else {
    const float2* rv = reinterpret_cast<const float2*>(raw);
#pragma unroll
    for (int jj = 0; jj < kKc / 2; ++jj) {
      const int idx = kc * (kKc / 2) + jj;
      const bool v = row_ok && ((a.mode == ANAL_C) ? (idx >= a.s0 && idx < a.s1) : (idx < a.n_omega));
      const float2 c = v ? rv[jj * kRowsCta + rr] : make_float2(0.f, 0.f);
      x[2 * jj] = c.x;
      x[2 * jj + 1] = c.y;
    }
  }
  // K-major core matrices: 4 consecutive K values of one row are one 16-byte vector
#pragma unroll
  for (int q = 0; q < kKc / 4; ++q) {
    float4 h, l;
    h.x = tc::to_tf32(x[4 * q]);
    h.y = tc::to_tf32(x[4 * q + 1]);
    h.z = tc::to_tf32(x[4 * q + 2]);
    h.w = tc::to_tf32(x[4 * q + 3]);
    l = make_float4(x[4 * q] - h.x, x[4 * q + 1] - h.y, x[4 * q + 2] - h.z, x[4 * q + 3] - h.w);
    const uint32_t o = tc::kmajor_offset(rr, 4 * q, kKc) / 4;
    *reinterpret_cast<float4*>(A_hi + o) = h;
    *reinterpret_cast<float4*>(A_lo + o) = l;
  }
}

// Accumulator columns [c0, c1) of row r (output columns coff + c): F stores, or FP64
// accumulator read-modify-writes, 32 columns per tensor-memory load, all loads of a
// group issued before use.
template <int W>
__device__ __forceinline__ void epilogue_cols(const ContractArgs& a, int64_t r, uint32_t tq, int cl, int coff,
                                              bool row_ok) {
  float v[32];
  if (W == 32) tc::tmem_ld32(tq + (uint32_t)cl, v);
  else tc::tmem_ld16(tq + (uint32_t)cl, v);
  if (!row_ok) return;
  const int c = coff + cl;
  if (a.mode == SYNTH_C) {
    float2* F = reinterpret_cast<float2*>(a.out);
#pragma unroll
    for (int q = 0; q < W; q += 2) {
      const int tau = (c + q) >> 1;
      if (tau < a.n_tau) __stcs(F + (int64_t)(a.tau0 + tau) * a.rows + r, make_float2(v[q], v[q + 1]));
    }
  } else if (a.mode == SYNTH_R) {
    float* F = reinterpret_cast<float*>(a.out);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int tau = c + q;
      if (tau < a.n_tau) __stcs(F + (int64_t)(a.tau0 + tau) * a.rows + r, v[q]);
    }
  } else {
    double2* __restrict__ acc = reinterpret_cast<double2*>(a.out);
    double2 old[W / 2];
#pragma unroll
    for (int q = 0; q < W / 2; ++q) {
      const int j = (c >> 1) + q;
      old[q] = j < a.n_omega ? __ldcs(acc + (int64_t)j * a.acc_stride + r) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < W / 2; ++q) {
      const int j = (c >> 1) + q;
      if (j < a.n_omega)
        __stcs(acc + (int64_t)j * a.acc_stride + r,
               make_double2(old[q].x + (double)v[2 * q], old[q].y + (double)v[2 * q + 1]));
    }
  }
}

__device__ __forceinline__ void epilogue_tile(const ContractArgs& a, int64_t r, uint32_t tq, int c0, int c1,
                                              int coff) {
  const bool row_ok = r < a.rows;
  int c = c0;
  for (; c + 32 <= c1; c += 32) epilogue_cols<32>(a, r, tq, c, coff, row_ok);
  if (c < c1) epilogue_cols<16>(a, r, tq, c, coff, row_ok);
}

__global__ void __launch_bounds__(kPipeThreads, 1) tc_contract_pipe_kernel(ContractArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* raw = smem;                                                     // [kRawRing][kRawBytes]
  float* sA = reinterpret_cast<float*>(smem + kRawRing * kRawBytes);             // [kAStages][hi, lo][..]
  float* sB = sA + kAStages * 2 * kAStageFloats;                                 // [kBRing][hi, lo][..]
  PipeBars* pb = reinterpret_cast<PipeBars*>(sB + kBRing * 2 * kBRingFloats);
  __shared__ uint32_t tbase;
  volatile int* abort_flag = &pb->abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < kRawRing; ++i) {
      tc::mbar_init(&pb->raw_full[i], 1);
      tc::mbar_init(&pb->raw_empty[i], 128);
    }
    for (int i = 0; i < kAStages; ++i) {
      tc::mbar_init(&pb->a_full[i], 128);
      tc::mbar_init(&pb->a_empty[i], 1);
    }
    for (int i = 0; i < kBRing; ++i) {
      tc::mbar_init(&pb->b_full[i], 1);
      tc::mbar_init(&pb->b_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&pb->acc_full[i], 1);
      tc::mbar_init(&pb->acc_empty[i], 256);
    }
    pb->abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tbase;
  const int chunks = a.K / kKc;
  const int64_t tiles = (a.rows + kRowsCta - 1) / kRowsCta;
  // Each row tile runs as one or two column sub-tiles of at most 256 columns; sub-tiles alternate
  // between the two accumulators, so the products of one overlap the epilogue of the previous one.
  const int nsub = a.N > 256 ? 2 : 1;

  if (warp == 12) {
    if (lane == 0) {  // producer of the long operand
      uint32_t g = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int64_t r0 = t * kRowsCta;
        const int nr = (int)min((int64_t)kRowsCta, a.rows - r0);
        for (int h = 0; h < nsub && ok; ++h) {   // the second sub-tile re-reads the rows from L2
          for (int kc = 0; kc < chunks; ++kc, ++g) {
            const uint32_t rs = g % kRawRing, ru = g / kRawRing;
            if (ru > 0 && !pwait(&pb->raw_empty[rs], (ru - 1) & 1, abort_flag)) { ok = false; break; }
            issue_raw(a, r0, nr, kc, raw + rs * kRawBytes, &pb->raw_full[rs]);
          }
        }
      }
      if (!ok) {
        pabort(pb, a.err);
        for (uint32_t q = 0; q < kRawRing && q < g; ++q) {  // the last copies land on their full barriers
          const uint32_t gg = g - 1 - q;
          tc::mbar_wait(&pb->raw_full[gg % kRawRing], (gg / kRawRing) & 1, kTries);
        }
      }
    }
  } else if (warp == 14) {
    if (lane == 0) {  // producer of the twiddle operand (the same chunks for every tile)
      uint32_t g = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        for (int h = 0; h < nsub && ok; ++h) {
          // rows [256 h, 256 h + nn) of a chunk are one contiguous run of 8-row core-matrix groups
          const int nn = h == 0 ? min(256, a.N) : a.N - 256;
          const uint32_t bytes = 4u * (uint32_t)nn * kKc;
          for (int kc = 0; kc < chunks; ++kc, ++g) {
            const uint32_t bs = g % kBRing, bu = g / kBRing;
            if (bu > 0 && !pwait(&pb->b_empty[bs], (bu - 1) & 1, abort_flag)) { ok = false; break; }
            float* B_hi = sB + bs * 2 * kBRingFloats;
            const float* bsrc = a.B + (size_t)kc * 2 * kBStageFloats + (size_t)h * 256 * kKc;
            tc::mbar_arrive_expect_tx(&pb->b_full[bs], 2 * bytes);
            tc::bulk_g2s(B_hi, bsrc, bytes, &pb->b_full[bs]);
            tc::bulk_g2s(B_hi + kBRingFloats, bsrc + kBStageFloats, bytes, &pb->b_full[bs]);
          }
        }
      }
      if (!ok) {
        pabort(pb, a.err);
        for (uint32_t q = 0; q < kBRing && q < g; ++q) {
          const uint32_t gg = g - 1 - q;
          tc::mbar_wait(&pb->b_full[gg % kBRing], (gg / kBRing) & 1, kTries);
        }
      }
    }
  } else if (warp == 13) {
    if (lane == 0) {  // MMA issuer
      uint32_t g = 0, tt = 0;
      bool ok = true;
      const uint32_t sbo = (kKc / 4) * 128;
      for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        for (int h = 0; h < nsub; ++h, ++tt) {
          const uint32_t buf = tt & 1, use = tt >> 1;
          if (use > 0 && !pwait(&pb->acc_empty[buf], (use - 1) & 1, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const int nn = h == 0 ? min(256, a.N) : a.N - 256;
          const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)nn);
          const uint32_t d = tmem + buf * 256u;
          for (int kc = 0; kc < chunks; ++kc, ++g) {
            const uint32_t as = g % kAStages, au = g / kAStages;
            const uint32_t bs = g % kBRing, bu = g / kBRing;
            if (!pwait(&pb->a_full[as], au & 1, abort_flag) || !pwait(&pb->b_full[bs], bu & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const char* A_hi = reinterpret_cast<const char*>(sA + as * 2 * kAStageFloats);
            const char* A_lo = A_hi + 4 * kAStageFloats;
            const char* B_hi = reinterpret_cast<const char*>(sB + bs * 2 * kBRingFloats);
            const char* B_lo = B_hi + 4 * kBRingFloats;
#pragma unroll
            for (int ks = 0; ks < kKc / 8; ++ks) {
              const uint64_t ah = tc::smem_desc(A_hi + ks * 256, 128, sbo);
              const uint64_t al = tc::smem_desc(A_lo + ks * 256, 128, sbo);
              const uint64_t bh = tc::smem_desc(B_hi + ks * 256, 128, sbo);
              const uint64_t bl = tc::smem_desc(B_lo + ks * 256, 128, sbo);
              tc::mma_tf32(d, ah, bh, idesc, kc > 0 || ks > 0);
              tc::mma_tf32(d, ah, bl, idesc, true);
              tc::mma_tf32(d, al, bh, idesc, true);
            }
            tc::mma_commit(&pb->a_empty[as]);
            tc::mma_commit(&pb->b_empty[bs]);
          }
          if (!ok) break;
          tc::mma_commit(&pb->acc_full[buf]);
        }
      }
      if (!ok) {
        pabort(pb, a.err);
        // every MMA issued so far completes before tensor memory is freed: a commit after them
        // completes the next phase of the current sub-tile's accumulator barrier
        tc::mma_commit(&pb->acc_full[tt & 1]);
        tc::mbar_wait(&pb->acc_full[tt & 1], (tt >> 1) & 1, kTries);
      }
    }
  } else if (warp < 4) {  // converters: one row each
    const int rr = tid;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int64_t r0 = t * kRowsCta;
      for (int h = 0; h < nsub && ok; ++h) {
        for (int kc = 0; kc < chunks; ++kc, ++g) {
          const uint32_t rs = g % kRawRing, ru = g / kRawRing;
          const uint32_t as = g % kAStages, au = g / kAStages;
          if (!pwait(&pb->raw_full[rs], ru & 1, abort_flag)) { ok = false; break; }
          if (au > 0 && !pwait(&pb->a_empty[as], (au - 1) & 1, abort_flag)) { ok = false; break; }
          float* A_hi = sA + as * 2 * kAStageFloats;
          convert_row(a, r0, kc, rr, raw + rs * kRawBytes, A_hi, A_hi + kAStageFloats);
          tc::fence_proxy_async_smem();
          mbar_arrive(&pb->a_full[as]);
          mbar_arrive(&pb->raw_empty[rs]);
        }
      }
    }
    if (!ok) pabort(pb, a.err);
  } else if (warp >= 4 && warp < 12) {  // epilogue: TMEM lane quadrant warp % 4, one half of the columns
    const int q = warp & 3;
    uint32_t tt = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      for (int h = 0; h < nsub; ++h, ++tt) {
        const uint32_t buf = tt & 1;
        if (!pwait(&pb->acc_full[buf], (tt >> 1) & 1, abort_flag)) { ok = false; break; }
        tc::tc_fence_after();
        const int nn = h == 0 ? min(256, a.N) : a.N - 256;
        const int half = round16c((nn + 1) / 2);
        const int c0 = warp < 8 ? 0 : half, c1 = warp < 8 ? half : nn;
        epilogue_tile(a, t * kRowsCta + 32 * q + lane, tmem + ((uint32_t)(32 * q) << 16) + buf * 256u, c0, c1,
                      256 * h);
        tc::tc_fence_before();
        mbar_arrive(&pb->acc_empty[buf]);
      }
    }
    if (!ok) pabort(pb, a.err);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
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

// The bulk copies of the pipelined kernel start on 16-byte boundaries and move
// whole 16-byte units: the long operand's base, its row stride and its row
// count must keep every copied row slice 16-byte aligned.
bool pipe_ok(const ContractArgs& a, rsv_operator op) {
  static const int env = [] {
    const char* e = getenv("RSV_CONTRACT_PIPE");
    return e != nullptr && e[0] == '0' ? 0 : 1;
  }();
  if (!env || op->sm_count <= 0) return false;
  if ((reinterpret_cast<uintptr_t>(a.src) & 15u) != 0) return false;
  if (a.mode == ANAL_R) return a.rows % 4 == 0;
  if (a.mode == ANAL_C) return a.rows % 2 == 0;
  return a.rows % 2 == 0 && a.src_stride % 2 == 0;
}

cudaError_t run(ContractArgs& a, const TileGeom& g, rsv_operator op) {
  const size_t bbytes = (size_t)(a.K / kKc) * 2 * kBStageFloats * sizeof(float);
  if (ensure(op->ws_tcb, bbytes) != RSV_OK) return cudaErrorMemoryAllocation;
  a.B = (const float*)op->ws_tcb.ptr;
  a.err = op->d_flag;
  const int64_t total = (int64_t)kMaxN * a.K;
  build_b_kernel<<<(unsigned)((total + 255) / 256), 256, 0, op->stream>>>(a, g, (const cpx<float>*)op->d_tw, op->d_pj,
                                                                          op->d_cw, (float*)op->ws_tcb.ptr);
  // the shared-memory opt-in is a per-device attribute: set it before every launch (cheap next
  // to a launch that moves gigabytes), so that any device and any thread gets it
  cudaError_t ae = cudaFuncSetAttribute(tc_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (ae == cudaSuccess)
    ae = cudaFuncSetAttribute(tc_contract_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeSmem);
  if (ae != cudaSuccess) return ae;
  const int64_t tiles = (a.rows + kRowsCta - 1) / kRowsCta;
  if (pipe_ok(a, op)) {
    const unsigned blocks = (unsigned)std::min<int64_t>(tiles, (int64_t)op->sm_count);
    tc_contract_pipe_kernel<<<blocks, kPipeThreads, kPipeSmem, op->stream>>>(a);
  } else {
    tc_contract_kernel<<<(unsigned)tiles, 256, kSmem, op->stream>>>(a);
  }
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
