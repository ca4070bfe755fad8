// Internal declarations shared by the CUDA translation units of libs2w.
// Nothing here is part of the public C ABI (include/s2w.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/s2w.h"

namespace s2w {

// Device status bits (latched in a device word, read back by s2w_sync).
enum : int {
  DEV_ERR_TIMEOUT_FULL = 1 << 0,   // consumer gave up waiting for a TMA stage
  DEV_ERR_TIMEOUT_EMPTY = 1 << 1,  // producer gave up waiting for a free stage
  DEV_ERR_TIMEOUT_MMA = 1 << 2,    // tensor-core pipeline wait gave up
  DEV_ERR_SHAPE = 1 << 3,          // a kernel saw an argument outside its limits
};

// Wall-clock bound on every spin-wait inside a kernel (nanoseconds).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Retransform stencil code for the adjoint (beside S2W_DT_BACKWARD / NONE):
// the transpose of the backward difference, u[n] = (w[n] - w[n+1]) / dt.
constexpr int kDtTranspose = 2;

// Storage codes of the resident spectra (same values as S2W_PREC_*).
enum Elem : int { EL_FP32 = 0, EL_BF16 = 1, EL_BF16_HILO = 2, EL_FP8 = 3, EL_FP32_HILO = 4 };

// Bytes of one complex entry of one stored array (the hi/lo kinds keep two).
__host__ __device__ inline int elem_complex_bytes(int el) {
  return (el == EL_FP32 || el == EL_FP32_HILO) ? 8 : (el == EL_FP8 ? 2 : 4);
}

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// PTX wrappers: shared-memory addresses, mbarriers, bulk async copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, for at most `limit_ns`
// (kWaitLimitNs by default).  On timeout, latch `code` into the device status
// word and return false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status, int code,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && globaltimer() - t0 > limit_ns) {
      atomicOr(status, code);
      return false;
    }
  }
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Bulk (non-tensor) asynchronous copy global -> this CTA's shared memory,
// completing `bytes` of transaction count on `bar`.  Both addresses must be
// 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// ---------------------------------------------------------------------------
// Host-side launchers implemented in the kernel translation units.
// All return cudaError_t of the launch (cudaGetLastError()).
// ---------------------------------------------------------------------------
// k_fft.cu
cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t st);
// Rows x[row][0..n_in) zero-padded to L = 2 Nt; bins l = 0..Nt of row `row`
// go to X[l * ld_l + (row / rows_a) * ld_a + row % rows_a].  lens (device,
// optional): row `row` uses only its first lens[row / rows_a] samples.
cudaError_t launch_rfft_rows(const float* x, long long rows, int n_in, int Nt, const float2* tw, float2* X,
                             long long ld_l, long long rows_a, long long ld_a, cudaStream_t st,
                             const int* lens = nullptr);
// Rows X[row][0..Nt] -> first Nt samples x[row][0..Nt) of the length-2Nt IFFT.
cudaError_t launch_irfft_rows(const float2* X, long long rows, int Nt, const float2* tw, float* x, cudaStream_t st);
// Retransform of `nb` ruptures (grid y): rupture y reads mhat + y * mhat_ld_b
// ([l][i] with bin stride ld_m) and writes either vhat + y * vhat_ld_b (FP32
// complex, bin stride ld_v) or, when vhat_bf is given, vhat_bf + y * vhat_ld_b
// (BF16 complex pairs, bin stride ld_v; with vhat_bf_lo also the low-order
// parts v - hi); seafloor (optional) + y * Ng * Nt.  n_alloc > 0 (with
// vhat_bf): rupture y writes rows 2y, 2y+1 of the conjugate-embedding B
// operand [l][n_alloc][ld_v] instead (vhat_ld_b unused).
cudaError_t launch_retransform(const float2* mhat, long long Ng, long long ld_m, int Nt, const float2* tw,
                               float inv_dt, int dt_mode, float2* vhat, long long ld_v, float* seafloor,
                               cudaStream_t st, int nb = 1, long long mhat_ld_b = 0, long long vhat_ld_b = 0,
                               __nv_bfloat162* vhat_bf = nullptr, __nv_bfloat162* vhat_bf_lo = nullptr,
                               int n_alloc = 0);
// q[b][o][n] from partials: Qhat[l] = sum_{s < nseg} part[b*s_b + l*s_l + s*s_s + o];
// the first n_keep (0: Nt) samples of the length-2Nt IFFT, rows n_keep apart.
cudaError_t launch_reduce_irfft(const float2* part, int B, int No, int nseg, int Nt, long long s_b, long long s_l,
                                long long s_s, const float2* tw, float* q, cudaStream_t st, int n_keep = 0);
// Partials part[l][s][e] (e < per): part[l][0][e] = sum over s < nseg, in
// increasing s (the order launch_reduce_irfft adds segments in).
cudaError_t launch_sum_chunks(float2* part, int Nb, int nseg, long long per, cudaStream_t st);
// Spectra X[l][r] (l < Nb, r < per_bin) times (1 - W_L^l) / dt, W_L^l = tw[l].
cudaError_t launch_scale_dt(float2* X, int Nb, long long per_bin, const float2* tw, float inv_dt, cudaStream_t st);
// r = q - d in place (B blocks of n_per_b floats); loss[b] = 0.5 sum r^2 (optional).
cudaError_t launch_residual(float* q, const float* d, int B, long long n_per_b, float* loss, cudaStream_t st);
cudaError_t launch_store_blocks(const float2* src, int Nb, long long n_per_l, int el, void* dst, void* dst_lo,
                                long long ld_dst_l, long long dst_off, cudaStream_t st);
cudaError_t launch_store_adjoint(const float2* src, int Nb, int No, long long nc, long long c0, int RL, int nseg,
                                 int el, void* dst, cudaStream_t st);
cudaError_t launch_fp8_store(const float2* spec, int Nb, long long rows, int Ns_pad, long long row0, long long Ng,
                             float* scale, int nblk, void* dst, cudaStream_t st);
// k_df.cu (FP32_HILO: spectra and intermediates as FP32 pairs hi + lo):
// tw[m] = exp(-2 pi i m / L) as (re hi, re lo, im hi, im lo), FP64-evaluated.
cudaError_t launch_twiddles_df(float4* tw, int L, cudaStream_t st);
// launch_rfft_rows with pair output (X hi, X_lo lo; same indexing).
cudaError_t launch_df_rfft_rows(const float* x, long long rows, int n_in, int Nt, const float4* tw, float2* X,
                                float2* X_lo, long long ld_l, long long rows_a, long long ld_a, cudaStream_t st,
                                const int* lens = nullptr);
// launch_retransform of one rupture with pairs in and out (dt_mode BACKWARD
// or NONE; seafloor optional, rounded to FP32).
cudaError_t launch_df_retransform(const float2* mhat, const float2* mhat_lo, long long Ng, long long ld_m, int Nt,
                                  const float4* tw, double inv_dt, int dt_mode, float2* vhat, float2* vhat_lo,
                                  long long ld_v, float* seafloor, cudaStream_t st);
// launch_reduce_irfft with pair partials (FP32 output).
cudaError_t launch_df_reduce_irfft(const float2* part, const float2* part_lo, int B, int No, int nseg, int Nt,
                                   long long s_b, long long s_l, long long s_s, const float4* tw, float* q,
                                   cudaStream_t st, int n_keep = 0);

// k_stream.cu: y[f] = sum_c rows[f][c] * x_vec(f)[c] for f < F, with
// x_vec(f) = x + (f / rows_per_vec) * x_stride.  Rows are contiguous,
// row_len complex entries each, row_len a multiple of 8 and <= 1024.
struct StreamArgs {
  const void* rows;
  const void* rows_lo;        // BF16 / FP32 hi/lo: the lo array (same layout), else nullptr
  long long F;
  int row_len;
  int el;                     // Elem
  const float2* x;
  const float2* x_lo;         // FP32_HILO: low-order parts of x (same layout)
  long long x_stride;         // complex entries between consecutive x vectors
  long long rows_per_vec;
  const float* scale;         // FP8: scale[(f / rows_per_vec) * nblk + (f % rows_per_vec) / 256]
  int nblk;
  float2* y;
  float2* y_lo;                // FP32_HILO: low-order parts of y
  int* status;
  unsigned long long wait_ns;  // bound of every wait (0: kWaitLimitNs)
  int fault_skip;              // test hook: 1 = the producer skips its first copy (consumers' waits run out)
};
cudaError_t launch_stream_dot(const StreamArgs& a, int num_sms, cudaStream_t st);

// k_stream.cu, transposed: y[u][c] = sum_{f in unit u} conj(rows[f][c]) w_f,
// unit u = chunk (u % nchunk) of Rc rows of group (u / nchunk) of G1 rows,
// w_f = w[w_base + (g / wa) * wb + (f - g G1)], g = f / G1 (times the FP8
// scale[g * nblk + (f - g G1) / 256] for FP8 rows).
struct StreamTArgs {
  const void* rows;
  const void* rows_lo;
  int el;
  int row_len;
  long long n_units;
  long long G1;
  int Rc, nchunk;
  const float2* w;
  long long w_base, wa, wb;
  const float* scale;
  int nblk;
  float2* y;
  int* status;
};
cudaError_t launch_stream_tdot(const StreamTArgs& a, int num_sms, cudaStream_t st);

// k_tc.cu: D = A B^T per bin on tensor cores (see the file comment).
struct TcArgs {
  int N;                  // MMA columns (multiple of 16; 256 or 512 above 256)
  int K;                  // reduction extent in BF16 elements
  int M_total;            // live rows of A per bin
  int Nb;                 // bins
  int m_tiles;            // ceil(M_total / 128)
  int n_kchunks;          // split of the K blocks into chunks (stage 2)
  int kblocks_per_chunk;  // 64-element K blocks per chunk
  int kb_off;             // first K block (a launch over one K range: chunk kc covers blocks
                          //   kb_off + kc kblocks_per_chunk ...)
  int acc_out;            // epi 0, FP32 out: add into out instead of storing (K ranges in turn)
  int stages;             // shared-memory ring depth
  int tmem_cols;          // power of two >= max(32, N)
  int epi;                // 0: out[l*ld_l + t*ld_t + row]; 1: out[((l*n_kchunks + kc)*M_total + row)*T + t]
  int T;                  // complex output columns (N / 2 live)
  float2* out;
  __nv_bfloat162* out_bf;  // epi 0: write BF16 pairs here instead of `out`
  long long ld_l, ld_t;
  const float* row_scale;  // optional per-(bin, 256-row block) scale
  int nblk;
  int a_lo;                // 1: A has a low-order BF16 part (second tensor map): adds A_lo B
  int b_lo;                // 1: B has a low-order BF16 part: adds A B_lo
  int a_fp8;               // 1: A is FP8 e4m3 (byte tensor map, row-major), widened to FP16 in shared memory;
                           //    needs row_scale; B is FP16 (launch_pack_b_f16) with its amax in b_amax
  const unsigned* b_amax;  // FP16 B operand: amax (float bits) that set its power-of-two scale
  int m_pair;              // 1: two M tiles per unit sharing each B tile (N <= 256, not FP8;
                           //    tmem_cols >= 2 N, stages from tc_stages_for(..., mt = 2))
  int b_half;              // 1: B holds rows 2t = (Re, -Im) of the plain embedding only, as rows
                           //    t < N / 2 (tensor map box N / 2 rows); four converter warps build
                           //    rows N / 2 + t = (Im, Re) per stage; output column t pairs
                           //    accumulator columns t and N / 2 + t.  BF16, one CTA per tile (or
                           //    M-tile pair), N <= 256 with N / 2 a multiple of 16, FP32 out
  int n_split;             // 2 (FP8 x hi + lo FP8 two-SM, N = 512): units of 256 columns, two
                           //    accumulators alternating in tensor memory; 128-element K blocks,
                           //    stages from tc_stages_pair(N / 2, 0, 4)
  int cta2;                // 1: two-SM MMAs, a CTA pair per M = 256 tile, each staging half of B
                           //    (N % 32 == 0, no m_pair; B box rows = min(N, 256) / 2,
                           //    K blocks tc_block_k(N, split, 1), stages from tc_stages_pair)
  int* status;
};
// bk = 64: 128-byte swizzle, K boxes of 64 BF16; bk = 32: 64-byte swizzle.
cudaError_t tc_encode_3d(CUtensorMap* out, const void* base, long long K, long long rows, long long nbatch,
                         long long row_pitch_elems, int box_rows, int bk = 64);
// K block (BF16 elements per swizzle row) and ring depth for N MMA columns
// with `terms` = 1 + a_lo + b_lo operand tiles beyond the first A and B
int tc_block_k(int N, int split = 0, int pair = 0);
int tc_stages_for(int N, int a_lo = 0, int b_lo = 0, int fp8 = 0, int mt = 1);
int tc_stages_pair(int N, int split, int fp8 = 0);
// Byte tensor map for FP8 A tiles: [nbatch][rows][K] bytes, box bk x box_rows, no swizzle
// (sw128 = 1: 128-byte swizzle, bk = 128; 2: 64-byte swizzle, bk = 64; for
// operands the MMAs read directly).
cudaError_t tc_encode_3d_u8(CUtensorMap* out, const void* base, long long K, long long rows, long long nbatch,
                            int box_rows, int bk, int sw128 = 0);
// tmA2 / tmB2: tensor maps of the low-order parts when a.a_lo / a.b_lo.
// col_scale (with a.a_fp8 and a.cta2): B is FP8 e4m3 too (launch_pack_b_f8),
// byte tensor maps with 128-byte swizzle and 128-byte K boxes, kind::f8f6f4
// MMAs; column t of bin l is scaled by col_scale[l * col_ld + t].  With
// col_scale and tmB2: B is hi + lo e4m3 parts (tmB, tmB2), two MMAs per K
// step; at N <= 256 with 64-byte swizzle and 64-byte K boxes for A and both
// B parts (a.stages from tc_stages_pair(N, 0, 3)), at N = 512 with
// a.n_split = 2 and 128-byte boxes.  (Kept out
// of TcArgs: a larger argument block costs every GEMM kernel registers.)
cudaError_t launch_tc_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcArgs& a, int num_sms,
                           cudaStream_t st, const CUtensorMap* tmA2 = nullptr, const CUtensorMap* tmB2 = nullptr,
                           const float* col_scale = nullptr, int col_ld = 0);
// B operand rows 2t / 2t+1 of dst[l][N_alloc][2 Kc] (BF16 pairs, hi and
// optional lo) from complex FP32 src[l*s_l + t*s_t + c], t < T, c < nc, at
// complex columns c0 + c; conj = 1 selects the embedding of conj(A) x;
// conj = 2 writes row 2t of the plain embedding, (Re, -Im), as row t only
// (the half-stored B of TcArgs::b_half).
cudaError_t launch_pack_b(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t, long long c0,
                          long long Kc, int N_alloc, int conj, void* hi, void* lo, cudaStream_t st);
// FP16 B operands: the power-of-two scale that keeps |x| * scale <= 2^14
// (inside the FP16 range with room to spare), and its inverse.
__device__ __forceinline__ float f16_scale(unsigned amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  if (!(amax > 0.f)) return 1.f;
  return exp2f(static_cast<float>(14 - static_cast<int>(ceilf(log2f(amax)))));
}
__device__ __forceinline__ float f16_unscale(unsigned amax_bits) { return 1.f / f16_scale(amax_bits); }
// Plain-embedding B operand as FP16 (k_pack_b layout, c0 = 0, no lo part):
// measures amax of the source first (amax: one device word), then packs x *
// f16_scale(amax).
// FP8 e4m3 B operand of the plain real embedding, rows 2t / 2t+1 of
// dst[l][N_alloc][2 Kc] bytes for t < n_rows / 2 (rows of t >= T zero, as is
// the K padding c >= nc), each pair of rows scaled by the power of two that
// brings its amax to at most 448 (e4m3's largest finite value), rounded to
// nearest even with saturation; col_scale[l * col_ld + t] = 1 / that scale.
// dst_lo (optional): the low-order parts, e4m3 of (scaled value - its e4m3
// rounding), in the same frame and layout.
cudaError_t launch_pack_b_f8(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t,
                             long long Kc, int N_alloc, int n_rows, float* col_scale, int col_ld, void* dst,
                             void* dst_lo, cudaStream_t st);
cudaError_t launch_pack_b_f16(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t,
                              long long Kc, int N_alloc, unsigned* amax, void* dst, cudaStream_t st);
// A operand dst[(l*rows_total + r0 + r)*Kc + c0 + c] (BF16 pairs, hi and
// optional lo) from complex FP32 src[l*s_l + r*s_r + c*s_c], r < rows, c < nc.
cudaError_t launch_pack_a(const float2* src, int Nb, int rows, long long nc, long long s_l, long long s_r,
                          long long s_c, long long rows_total, long long r0, long long c0, long long Kc, void* hi,
                          void* lo, cudaStream_t st);
// Retransform of Bs ruptures as one GEMM per 128-signal tile (see k_tc.cu):
// reads mhat[l*ld_l + b*ld_b + i], writes vhat[l*vld_l + b*vld_b + i] (BF16
// pairs); tmT: T[n][k], 2 Nt x 2 Nt BF16, K-major.  32 <= Nt <= 256.
struct TcRtArgs {
  const __nv_bfloat162* mhat_bf;  // seafloor spectra, BF16 (re, im) pairs [l][b][i]
  const float2* mhat32;           // split: seafloor spectra, FP32 (same indexing)
  long long ld_l, ld_b;
  int Ng, Bs, Nt;
  __nv_bfloat162* vhat;
  __nv_bfloat162* vhat_lo;        // split: low-order parts of vhat
  long long vld_l, vld_b;
  long long conj_row;             // > 0: write the conjugate-embedding B operand: (Re, Im) at the
                                  // output position and (Im, -Re) conj_row entries further
  int ra, rt;                     // ring depths: A (one slot per fill warp) and T (set by the launcher)
  int* status;
};
// tmT2 (split): tensor map of T's low-order part; T maps then use 32-element
// K boxes (64-byte swizzle), else 64 (128-byte swizzle).  tmTp (BF16 only):
// a map of the same T with boxes of half the rows (min(2 Nt, 256) / 2),
// which selects two-SM tiles when the grid spans at least two M tiles.
cudaError_t launch_tc_retransform(const CUtensorMap& tmT, const CUtensorMap* tmT2, const TcRtArgs& a, int num_sms,
                                  cudaStream_t st, const CUtensorMap* tmTp = nullptr);

}  // namespace s2w
