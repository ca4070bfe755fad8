// Tensor-core per-bin contractions for rupture batches (Alg. 2 step 3 with
// many right-hand sides): tcgen05.mma with FP32 accumulators in tensor
// memory (kind::f16 for BF16 / FP16 operands, kind::f8f6f4 for e4m3 x e4m3),
// operands staged by TMA with 128-byte (or 64-byte) swizzle.  Two GEMM
// bodies: tc_gemm_body, one CTA per 128-row tile (optionally two tiles per
// unit sharing each B tile), and tc_gemm2_body, the two-SM form
// (cta_group::2: a CTA pair per 256-row tile, each staging half of B).  Every
// CTA issues its own TMA loads of the tiles it uses; tiles shared by
// several CTAs are served from L2.
// The retransform between the stages is a GEMM too (k_tc_retransform).
//
// Complex products run as one real GEMM per bin through a real embedding that
// never duplicates the streamed operand A:
//   A[r][2c] = Re a_rc, A[r][2c+1] = Im a_rc                  (K-major, as stored)
//   B[2t][2c] = Re x_ct,  B[2t][2c+1] = -Im x_ct               (row 2t: real part)
//   B[2t+1][2c] = Im x_ct, B[2t+1][2c+1] = Re x_ct             (row 2t+1: imaginary part)
//   D = A B^T  =>  D[r][2t] + i D[r][2t+1] = sum_c a_rc x_ct.
// Stage 1: A = Ghat_l (rows = grid points, c = subfault), x = shat_l over the
//          batch (t = rupture);  D -> mhat[l][b][i].
// Stage 2: A = vhat_l (rows = ruptures, c = grid point), B built from Phat_l
//          (t = observation);  split over chunks of grid points, D -> partials.
//
// Warp roles (576 threads, one CTA per SM, persistent over work units):
//   warp 0  one lane issues TMA loads into a ring of K-block stages;
//   warp 1  allocates tensor memory; one lane issues tcgen05.mma and commits;
//   warps 2-17 epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//              lanes 32 (w % 4) .. +31, i.e. tile rows, and every fourth
//              64-column chunk), scale, store.  Four warps per lane quadrant
//              cut the time the MMAs wait for the accumulator to drain
//              (with N = 512 it fills tensor memory, so it cannot be
//              double-buffered); FP8 kernels keep two per quadrant.  The
//              two-SM FP8 x (hi + lo FP8) kernel at N = 512 instead splits
//              the columns into two 256-column units (n_split) whose
//              accumulators alternate, so the drain overlaps the MMAs.
//   warps 10-13 (448-thread kernels: FP8 A widened to FP16, and the
//              stage-2 GEMM on the half-stored adjoint operand) complete
//              each stage in shared memory before the MMAs read it; these
//              kernels keep two epilogue warps per quadrant (warps 2-9).
// Every mbarrier wait is bounded (s2w_internal.cuh); on expiry a status bit
// is latched and the CTA drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "s2w_internal.cuh"

namespace s2w {

namespace {

// epilogue warps per TMEM lane quadrant (warps 2 .. 2 + 4 EPW - 1); the FP8
// kernels keep fewer, their 4 converter warps need the registers
constexpr int kEpw = 4;
constexpr int kEpwF8 = 2;
constexpr int kTcThreads = 32 * (2 + 4 * kEpw);         // warps: 0 TMA producer, 1 MMA, then the epilogue
constexpr int kTcThreadsF8 = 32 * (2 + 4 * kEpwF8) + 128;  // FP8 A: + 4 warps widen the A tiles to FP16
constexpr int kBlockM = 128;
constexpr int kSmemBudget = 200 * 1024;
constexpr int kSmemOptInLimit = 227 * 1024;  // opt-in dynamic shared memory per CTA

__device__ __forceinline__ void tma_load_3d(void* sdst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(sdst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Arrive once on `bar` when every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 lanes x 16 columns of 32-bit accumulators: thread t of the warp gets
// columns [col, col + 16) of TMEM lane (lane base + t).  The load and its
// wait are one asm statement, so no use of the outputs can be scheduled
// before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Same for 64 columns in one load (one wait per 64 accumulators).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, "
      "%38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, "
      "%60, %61, %62, %63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 64; ++k) v[k] = __uint_as_float(r[k]);
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row core-matrix groups 1024 bytes
// apart (stride byte offset), tile base 1024-byte aligned; advancing along K
// inside the swizzle row is a plain byte offset of the start address.
template <int BK>
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
  // BK = 64: rows of 128 B, 128-byte swizzle; BK = 32: rows of 64 B, 64-byte swizzle
  constexpr uint32_t sbo = 8 * BK * 2;
  constexpr uint64_t layout = BK == 64 ? 2 : 4;
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                  // leading byte offset (unused here)
  d |= static_cast<uint64_t>(sbo >> 4) << 32;           // stride byte offset (8-row groups)
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version (tcgen05)
  d |= layout << 61;                                    // swizzle mode
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// Same with FP16 A and B (the A / B format fields left at 0 = F16).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// Epilogue of one 128 x N accumulator at TMEM address tbase (this warp's lane
// quadrant): the thread owning tile row `row` scales its columns and stores
// them, column pair (2t, 2t+1) as complex column t < T, to
//   epi 0: out[l ld_l + t ld_t + row]  (BF16 pairs when out_bf is set),
//   epi 1: out[((l n_kchunks + kc) M_total + row) T + t].
// Epilogue warp group g of EPW takes the 64-column chunks g, g + EPW, ...
// and the 16-column chunks of the tail likewise.  Every lane runs the
// tcgen05.ld (warp-collective); rows that are not live store nothing.
// CS: per-column scales of this bin (FP8 B operand), cs[t].
template <int NC, bool CS>
__device__ __forceinline__ void tc_store_cols(const TcArgs& a, const float* v, int t0, long long obase, long long ld,
                                              bool bf, float scale, const float* cs, int T) {
  const int nt = T - t0;  // live complex columns from t0 (all NC when >= NC)
  if (bf) {
    __nv_bfloat162* p = a.out_bf + obase + t0 * ld;
#pragma unroll
    for (int k = 0; k < NC; ++k)
      if (k < nt) {
        const float sk = CS ? scale * cs[t0 + k] : scale;
        p[k * ld] = __floats2bfloat162_rn(v[2 * k] * sk, v[2 * k + 1] * sk);
      }
  } else {
    float2* p = a.out + obase + t0 * ld;
#pragma unroll
    for (int k = 0; k < NC; ++k)
      if (k < nt) {
        const float sk = CS ? scale * cs[t0 + k] : scale;
        float2 o = make_float2(v[2 * k] * sk, v[2 * k + 1] * sk);
        if (a.acc_out) o = cadd(p[k * ld], o);  // K chunk after the first: add into the output
        p[k * ld] = o;
      }
  }
}

template <int EPW, bool CS = false>
__device__ __forceinline__ void tc_epilogue_tile(const TcArgs& a, uint32_t tbase, int N, int g, int l, int kc,
                                                 int row, bool live, float scale, const float* cs = nullptr,
                                                 int t_off = 0) {
  const bool bf = a.epi == 0 && a.out_bf != nullptr;
  const long long ld = a.epi == 0 ? a.ld_t : 1;
  const long long obase =
      (a.epi == 0 ? static_cast<long long>(l) * a.ld_l + row
                  : ((static_cast<long long>(l) * a.n_kchunks + kc) * a.M_total + row) * a.T) +
      static_cast<long long>(t_off) * ld;
  const int T = a.T - t_off;  // live complex columns of this accumulator
  if (CS) cs += t_off;
  const int n64 = N / 64 * 64;
  for (int c0 = 64 * g; c0 < n64; c0 += 64 * EPW) {
    float v[64];
    tmem_ld64(tbase + c0, v);
    if (live && c0 / 2 < T) tc_store_cols<32, CS>(a, v, c0 / 2, obase, ld, bf, scale, cs, T);
  }
  for (int c0 = n64 + 16 * g; c0 < N; c0 += 16 * EPW) {
    float v[16];
    tmem_ld16(tbase + c0, v);
    if (live && c0 / 2 < T) tc_store_cols<8, CS>(a, v, c0 / 2, obase, ld, bf, scale, cs, T);
  }
}

// Epilogue with a half-stored B (TcArgs::b_half): accumulator columns t and
// N / 2 + t hold the real and imaginary parts of complex column t (B rows
// t = (Re, -Im) and N / 2 + t = (Im, Re) of one column of the embedding).
// Group g of EPW takes the 16-column chunks g, g + EPW, ... of the first
// half; N / 2 is a multiple of 16.  FP32 pairs out (epi 0 or 1).
template <int EPW>
__device__ __forceinline__ void tc_epilogue_half(const TcArgs& a, uint32_t tbase, int N, int g, int l, int kc,
                                                 int row, bool live, float scale) {
  const int nh = N / 2;
  const long long ld = a.epi == 0 ? a.ld_t : 1;
  const long long obase = a.epi == 0
                              ? static_cast<long long>(l) * a.ld_l + row
                              : ((static_cast<long long>(l) * a.n_kchunks + kc) * a.M_total + row) * a.T;
  for (int t0 = 16 * g; t0 < nh; t0 += 16 * EPW) {
    float re[16], im[16];
    tmem_ld16(tbase + t0, re);
    tmem_ld16(tbase + nh + t0, im);
    if (!live || t0 >= a.T) continue;
    float2* p = a.out + obase + t0 * ld;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (t0 + k < a.T) {
        float2 o = make_float2(re[k] * scale, im[k] * scale);
        if (a.acc_out) o = cadd(p[k * ld], o);
        p[k * ld] = o;
      }
  }
}

// Row t of the embedding's second half from row t of the first: each BF16
// pair (a, b) becomes (-b, a) -- the halves swapped and the sign bit of the
// new low half flipped (exact).
__device__ __forceinline__ unsigned rot_pair_bf16(unsigned w) { return __funnelshift_l(w, w, 16) ^ 0x8000u; }

// Widens row t of an FP8 e4m3 A tile (BK bytes at src, as TMA wrote it
// without swizzle) exactly to FP16 (one cvt per pair) and stores the BK * 2
// bytes at dst in the TMA swizzle pattern of a BK-element K-major row
// (128 B: chunk ^ (row & 7); 64 B: chunk ^ ((row >> 1) & 3)).
template <int BK>
__device__ __forceinline__ void widen_fp8_row(const unsigned char* src_row, unsigned char* dst, int t) {
  const uint4* src = reinterpret_cast<const uint4*>(src_row);
#pragma unroll
  for (int c = 0; c < BK / 16; ++c) {  // 16 FP8 in -> two 16-byte FP16 chunks out
    const int cc = (c + t) % (BK / 16);  // staggered start: fewer bank conflicts
    const uint4 w = src[cc];
    const unsigned ww[4] = {w.x, w.y, w.z, w.w};
    unsigned o[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __half2_raw hr =
            __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>((ww[k] >> (16 * h)) & 0xffffu), __NV_E4M3);
        o[2 * k + h] = static_cast<unsigned>(hr.x) | (static_cast<unsigned>(hr.y) << 16);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ch = 2 * cc + h;
      const int sw = BK == 64 ? (ch ^ (t & 7)) : (ch ^ ((t >> 1) & 3));
      *reinterpret_cast<uint4*>(dst + (sw << 4)) = make_uint4(o[4 * h], o[4 * h + 1], o[4 * h + 2], o[4 * h + 3]);
    }
  }
}

// One ring of K-block stages, each holding the A tile and the B tile of the
// same K block (loaded together, released together).
// Split precision (a_lo / b_lo): an operand stored as hi + lo BF16 parts has
// both parts in every stage, and each K step issues A B, then A B_lo and/or
// A_lo B into the same FP32 accumulator (the A_lo B_lo term, ~2^-18
// relative, is dropped).
// MODE: 0 BF16 operands; 1 split (hi/lo parts of both operands); 2 FP8 e4m3
// A: TMA brings the FP8 tile (row-major, one byte per K element) into a
// staging slot of the stage, warps 10-13 widen it exactly to FP16 (one
// cvt per pair) into the swizzled A slot and signal `aready`; the MMAs take
// FP16 A and B (B packed as FP16 with a power-of-two scale from its amax);
// the per-(bin, 256-row) scale and the B scale are undone in the epilogue.
// 5 BF16 with B stored as its first N / 2 rows (TcArgs::b_half): TMA loads
// those into the first half of the stage's B tile, warps 10-13 write the
// second half (rot_pair_bf16 of each word) and signal `aready`, and the
// epilogue pairs accumulator columns t and N / 2 + t (tc_epilogue_half).
// Each MODE is its own instantiation and kernel, so the plain kernel carries
// none of the other modes' code.
// MT = 2 (N <= 256, not FP8): a unit takes two adjacent M tiles
// that share every B tile, with one accumulator each (2N TMEM columns): A
// gets two thirds of each stage instead of half at N = 128, and B is read
// from L2 once per two tiles.
template <int BK, int MODE, int MT = 1>
__device__ __forceinline__ void tc_gemm_body(const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmA2,
                                             const CUtensorMap* tmB2, const TcArgs& a) {
  static_assert(MT == 1 || MODE != 2, "M-tile pairs: not with FP8 A");
  constexpr bool SPLIT = MODE == 1;
  constexpr bool F8 = MODE == 2;
  constexpr bool BH = MODE == 5;    // B stored as its first N / 2 rows (TcArgs::b_half)
  constexpr bool CONV = F8 || BH;   // 4 converter warps complete each stage
  constexpr int EPW = CONV ? kEpwF8 : kEpw;
  constexpr int kEpiWarps = 4 * EPW;
  constexpr int kConvWarp0 = 2 + kEpiWarps;  // first of the 4 converter warps
  constexpr int kStg = F8 ? kBlockM * BK : 0;  // FP8 staging bytes per stage
  constexpr int kA = kBlockM * BK * 2;
  constexpr int a_tile = kA * (SPLIT ? 2 : 1);  // one M tile's A (+ A_lo) bytes per stage
  const long long cid = static_cast<long long>(blockIdx.x);
  const long long ncl = static_cast<long long>(gridDim.x);
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int N = a.N;
  const int b_bytes = N * BK * 2;
  constexpr int a_all = a_tile * MT;                   // A (+ A_lo) bytes per stage, all M tiles
  const int stage_bytes = a_all + b_bytes * (SPLIT ? 2 : 1) + kStg;
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* aready = empty + S;  // F8 / BH: the stage completed (count 4 converter warps)
  uint64_t* acc_full = aready + (CONV ? S : 0);
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + 1);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nk_total = (a.K + BK - 1) / BK;
  const int mtg = (a.m_tiles + MT - 1) / MT;  // M-tile groups (one per unit)
  const long long units = static_cast<long long>(a.Nb) * mtg * a.n_kchunks;
  const int n_mma = N > 256 ? N / 256 : 1;
  const int n_mma_cols = N > 256 ? 256 : N;
  // FP8 A is widened to FP16 (one conversion per pair, exact); B is FP16 too
  const uint32_t idesc = F8 ? idesc_f16(kBlockM, n_mma_cols) : idesc_bf16(kBlockM, n_mma_cols);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
      if (CONV) mbar_init(aready + s, 4);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_holder, a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  auto unit_coords = [&](long long u, int& l, int& mt, int& kc) {
    kc = static_cast<int>(u % a.n_kchunks);
    const long long r = u / a.n_kchunks;
    mt = static_cast<int>(r % mtg) * MT;  // first M tile of the unit
    l = static_cast<int>(r / mtg);
  };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (long long u = cid; u < units && ok; u += ncl) {
        int l, mt, kc;
        unit_coords(u, l, mt, kc);
        const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
        const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          if (it >= S && !mbar_wait_bounded(empty + s, ((it / S) - 1) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * stage_bytes;
          // F8: the A slot is not TMA's; BH: nor the second half of B
          mbar_arrive_expect_tx(full + s, stage_bytes - (F8 ? kA : 0) - (BH ? b_bytes / 2 : 0));
          if constexpr (F8) {
            tma_load_3d(sa + a_all + b_bytes, tmA, kb * BK, mt * kBlockM, l, full + s);
          } else {
            // rows past the last M tile read as zeros (TMA fill); their outputs are never stored
#pragma unroll
            for (int j = 0; j < MT; ++j) {
              tma_load_3d(sa + j * a_tile, tmA, kb * BK, (mt + j) * kBlockM, l, full + s);
              if constexpr (SPLIT) tma_load_3d(sa + j * a_tile + kA, tmA2, kb * BK, (mt + j) * kBlockM, l, full + s);
            }
          }
          auto load_b = [&](const CUtensorMap* tb, unsigned char* sb) {
            for (int c = 0; c < n_mma; ++c)
              tma_load_3d(sb + c * n_mma_cols * BK * 2, tb, kb * BK, c * n_mma_cols, l, full + s);
          };
          if constexpr (BH)
            tma_load_3d(sa + a_all, tmB, kb * BK, 0, l, full + s);  // box: the N / 2 stored rows
          else
            load_b(tmB, sa + a_all);
          if constexpr (SPLIT) load_b(tmB2, sa + a_all + b_bytes);
        }
      }
      for (int kk = (it > S ? it - S : 0); kk < it; ++kk)
        mbar_wait_bounded(full + kk % S, (kk / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL);
      // the last stages must also have been released by the MMAs before the
      // CTA tears down
      for (int kk = (it > S ? it - S : 0); kk < it; ++kk)
        mbar_wait_bounded(empty + kk % S, (kk / S) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, acc_it = 0;
      bool ok = true;
      for (long long u = cid; u < units && ok; u += ncl) {
        int l, mt, kc;
        unit_coords(u, l, mt, kc);
        const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
        const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
        if (acc_it > 0 && !mbar_wait_bounded(acc_empty, (acc_it - 1) & 1, a.status, DEV_ERR_TIMEOUT_MMA)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          if (!mbar_wait_bounded(CONV ? aready + s : full + s, (it / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * stage_bytes);
          const uint32_t sb = sa + a_all;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
#pragma unroll
            for (int j = 0; j < MT; ++j) {  // accumulator j at TMEM columns j N ..
              const uint32_t aoff = j * a_tile + k * 32;
              const uint64_t ad = sdesc_sw<BK>(sa + aoff);
              for (int c = 0; c < n_mma; ++c) {
                const uint32_t boff = c * n_mma_cols * BK * 2 + k * 32;
                const uint64_t bd = sdesc_sw<BK>(sb + boff);
                const uint32_t dcol = tmem + j * N + c * n_mma_cols;
                tc_mma_bf16(dcol, ad, bd, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
                if constexpr (SPLIT) {
                  tc_mma_bf16(dcol, ad, sdesc_sw<BK>(sb + b_bytes + boff), idesc, 1u);
                  tc_mma_bf16(dcol, sdesc_sw<BK>(sa + aoff + kA), bd, idesc, 1u);
                }
              }
            }
          }
          tc_commit(empty + s);
        }
        if (!ok) break;
        tc_commit(acc_full);
        ++acc_it;
      }
      // the epilogue consumes the last accumulator; wait for it before teardown
      if (acc_it > 0) mbar_wait_bounded(acc_empty, (acc_it - 1) & 1, a.status, DEV_ERR_TIMEOUT_MMA);
    }
  } else if (CONV && warp >= kConvWarp0) {
    // converter warps.  F8: thread t widens row t of each FP8 A tile.  BH:
    // the B tile's second half, row by row from the first (rows N / 2 + r
    // and r share the 128-byte swizzle phase, N / 2 being a multiple of 8,
    // so the bytes copy straight across), 16 bytes per thread and step
    const int t = threadIdx.x - 32 * kConvWarp0;
    int it = 0;
    bool ok = true;
    for (long long u = cid; u < units && ok; u += ncl) {
      int l, mt, kc;
      unit_coords(u, l, mt, kc);
      const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
      const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % S;
        if (!mbar_wait_bounded(full + s, (it / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL)) {
          ok = false;
          break;
        }
        unsigned char* sa = smem + s * stage_bytes;
        if constexpr (F8) {
          widen_fp8_row<BK>(sa + a_all + b_bytes + t * BK, sa + t * (BK * 2), t);
        } else {
          const uint4* src = reinterpret_cast<const uint4*>(sa + a_all);
          uint4* dst = reinterpret_cast<uint4*>(sa + a_all + b_bytes / 2);
          for (int i = t; i < b_bytes / 32; i += 128) {
            const uint4 w = src[i];
            dst[i] = make_uint4(rot_pair_bf16(w.x), rot_pair_bf16(w.y), rot_pair_bf16(w.z), rot_pair_bf16(w.w));
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(aready + s);
      }
    }
  } else {
    // epilogue warps 2 .. 2 + kEpiWarps - 1
    const int q = warp & 3;          // TMEM lane quadrant this warp may access
    const int g = (warp - 2) >> 2;   // column group of the quadrant
    int acc_it = 0;
    for (long long u = cid; u < units; u += ncl) {
      int l, mt, kc;
      unit_coords(u, l, mt, kc);
      if (!mbar_wait_bounded(acc_full, acc_it & 1, a.status, DEV_ERR_TIMEOUT_MMA)) break;
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < MT; ++j) {
        const int row = (mt + j) * kBlockM + q * 32 + lane;
        const uint32_t tbase = tmem + j * N + (static_cast<uint32_t>(q * 32) << 16);
        const bool live = row < a.M_total && mt + j < a.m_tiles;
        float scale = 1.f;
        if (a.row_scale != nullptr && live) scale = a.row_scale[static_cast<long long>(l) * a.nblk + row / 256];
        if (a.b_amax != nullptr) scale *= f16_unscale(*a.b_amax);  // undo the FP16 B operand's power-of-two scale
        if constexpr (BH)
          tc_epilogue_half<EPW>(a, tbase, N, g, l, kc, row, live, scale);
        else
          tc_epilogue_tile<EPW>(a, tbase, N, g, l, kc, row, live, scale);
      }  // M tiles of the unit
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      ++acc_it;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm_body<BK, 0>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm_body<BK, 0, 2>(&tmA, &tmB, nullptr, nullptr, a);
}

// BF16 operands with B stored as the first half of its rows (b_half): the
// stage-2 GEMM on the adjoint spectra stored once, (Re, -Im) per observation.
template <int BK>
__global__ void __launch_bounds__(kTcThreadsF8, 1)
    k_tc_gemm_h(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm_body<BK, 5>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreadsF8, 1)
    k_tc_gemm_pair_h(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const TcArgs a) {
  tc_gemm_body<BK, 5, 2>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm_split_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                         const TcArgs a) {
  tc_gemm_body<BK, 1, 2>(&tmA, &tmB, &tmA2, &tmB2, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreadsF8, 1)
    k_tc_gemm_f8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm_body<BK, 2>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm_split(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                    const TcArgs a) {
  tc_gemm_body<BK, 1>(&tmA, &tmB, &tmA2, &tmB2, a);
}

// ---------------------------------------------------------------------------
// Two-SM form (tcgen05 cta_group::2).  A cluster of two CTAs computes one
// M = 256 tile: rank 0 holds A rows [0, 128) of it, rank 1 rows [128, 256).
// Each N <= 256 slice c of the B tile is split between the pair, rank r
// staging columns [c 256 + r h, + h) with h = slice / 2.  One thread of rank 0
// issues M = 256 MMAs that read both CTAs' shared memory and leave each
// CTA's 128 accumulator rows in its own tensor memory.  Per CTA and K step
// this halves the B bytes staged and read against one CTA per M tile.
// Barriers: full[s] is used in rank 0 only (the TMA loads of both CTAs
// complete on it); empty[s] and acc_full exist in both and receive the MMA
// commits as mbarrier arrives in both CTAs (tcgen05.commit with a CTA mask:
// an arrive, no data moves); acc_empty in rank 0 counts the epilogue warps of
// both CTAs (rank 1's arrive remotely).  Every tcgen05 allocation, MMA and
// commit of the kernel uses cta_group::2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// TMA load into this CTA's shared memory that completes on the mbarrier at
// cluster address `bar` (this CTA's or its pair peer's).
__device__ __forceinline__ void tma_load_3d_pair(void* sdst, const CUtensorMap* tm, int c0, int c1, int c2,
                                                 uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(smem_u32(sdst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// mbar_wait_bounded with cluster-scope acquire (arrivals from the peer CTA).
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded_cl(uint64_t* bar, uint32_t parity, int* status, int code) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    if ((it & 255u) == 0u && globaltimer() - t0 > kWaitLimitNs) {
      atomicOr(status, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tmem_alloc2(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish2() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Arrive once on `bar` in each CTA of the pair whose bit is set in `mask` when
// this thread's issued MMAs complete (an mbarrier arrive only).
__device__ __forceinline__ void tc_commit2_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void tc_mma2_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Same with 8-bit operands (kind::f8f6f4; both e4m3 with the f16 instruction
// descriptor's zero type fields), K = 32 per instruction.
__device__ __forceinline__ void tc_mma2_f8f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// MODE 0: BF16 operands; 1: split (A, A_lo, B, B_lo; three MMAs per K step);
// 2: FP8 e4m3 A widened to FP16 in shared memory by 4 converter warps per
// CTA, FP16 B.  Stage layout per CTA: A [A_lo] B-halves [B_lo-halves]
// [FP8 staging].  FP8: each CTA's staging load completes on its own full[s],
// and rank 0's full[s] also takes both CTAs' B halves; the converters of
// both CTAs then arrive on rank 0's aready[s], which the MMAs wait for.
// 3: FP8 e4m3 A and B (kind::f8f6f4, no widening): BK counts bytes =
// elements, K = 32 per MMA; the per-(bin, 256-row) A scales and per-(bin,
// column) B scales are applied in the epilogue.  4: the same with B as hi +
// lo e4m3 parts, two MMAs per K step.  MODE 4 with a.n_split = 2
// (N = 512): a unit is one 256-column half of an M = 256 tile (the two
// halves are adjacent units, taken by neighbouring CTA pairs at about the
// same time, so A comes from HBM about once), its
// accumulator one of two alternating 256-column slots of tensor memory: the
// epilogue drains one while the MMAs fill the other (with one 512-column
// accumulator the MMAs waited ~20 % of each unit for the drain).  MODE 3
// reads half the B bytes per K step, and there the second A read of each
// tile cost more than the overlap gained (measured), so it keeps N = 512.
template <int BK, int MODE>
__device__ __forceinline__ void tc_gemm2_body(const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmA2,
                                              const CUtensorMap* tmB2, const TcArgs& a,
                                              const float* col_scale = nullptr, int col_ld = 0) {
  constexpr bool SPLIT = MODE == 1;
  constexpr bool F8 = MODE == 2;
  constexpr bool F8F8 = MODE == 3 || MODE == 4;
  constexpr bool BLO = MODE == 4;         // FP8 B as hi + lo e4m3 parts: two MMAs per K step
  constexpr int ES = F8F8 ? 1 : 2;        // operand bytes per element in shared memory
  constexpr int BKB = BK * ES;            // bytes per K-major row of a k-block
  constexpr int KI = F8F8 ? 32 : 16;      // K per MMA instruction (32 bytes either way)
  constexpr int EPW = F8 ? kEpwF8 : kEpw;
  constexpr int kEpiWarps = 4 * EPW;
  constexpr int kConvWarp0 = 2 + kEpiWarps;
  constexpr int kA = kBlockM * BKB;
  constexpr int kStg = F8 ? kBlockM * BK : 0;  // FP8 staging bytes per stage
  const uint32_t crank = cluster_ctarank();
  const bool lead = crank == 0;
  const long long cid = static_cast<long long>(cluster_id_x());
  const long long ncl = static_cast<long long>(cluster_count_x());
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int N = a.N;
  // F8F8 with n_split = 2 (N = 512): a unit takes one 256-column half of the
  // columns, and two such accumulators alternate in tensor memory, so the
  // MMAs of the next unit run while the epilogue drains the last one
  const int NS = (BLO && a.n_split == 2) ? 2 : 1;
  const int NU = N / NS;       // accumulator columns per unit
  const int AS = NS;           // accumulators in tensor memory
  const int n_mma = NU > 256 ? NU / 256 : 1;
  const int n_mma_cols = NU > 256 ? 256 : NU;
  const int hrows = n_mma_cols / 2;  // B rows this CTA stages per MMA slice
  const int hb = hrows * BKB;
  const int bh_bytes = n_mma * hb;
  const int a_bytes = kA * (SPLIT ? 2 : 1);
  const int b_all = bh_bytes * ((SPLIT || BLO) ? 2 : 1);
  const int stage_bytes = a_bytes + b_all + kStg;
  const int S = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* aready = empty + S;  // F8, rank 0: both CTAs' A slots widened
  constexpr int kAccBars = BLO ? 2 : 1;  // hi + lo B may alternate two accumulators
  uint64_t* acc_full = aready + (F8 ? S : 0);
  uint64_t* acc_empty = acc_full + kAccBars;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + kAccBars);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nk_total = (a.K + BK - 1) / BK;
  const int mpairs = (a.m_tiles + 1) / 2;
  const long long units = static_cast<long long>(a.Nb) * mpairs * NS * a.n_kchunks;
  // FP16 (F8) and e4m3 (F8F8, kind::f8f6f4) both encode as type 0
  const uint32_t idesc = (F8 || F8F8) ? idesc_f16(2 * kBlockM, n_mma_cols) : idesc_bf16(2 * kBlockM, n_mma_cols);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
      if (F8) mbar_init(aready + s, 8);  // 4 converter warps of each CTA
    }
    for (int s = 0; s < kAccBars; ++s) {
      mbar_init(acc_full + s, 1);
      mbar_init(acc_empty + s, 2 * kEpiWarps);
    }
    fence_mbar_init();
  }
  if (warp == 1) {  // one warp of each CTA allocates the pair's tensor memory together
    tmem_alloc2(tmem_holder, a.tmem_cols);
    tmem_relinquish2();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers and tensor memory exist before any load or MMA
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  auto unit_coords = [&](long long u, int& l, int& mt, int& nh, int& kc) {
    kc = static_cast<int>(u % a.n_kchunks);
    long long r = u / a.n_kchunks;
    nh = static_cast<int>(r % NS);  // column half (n_split)
    r /= NS;
    mt = static_cast<int>(r % mpairs) * 2 + static_cast<int>(crank);  // this CTA's M tile
    l = static_cast<int>(r / mpairs);
  };

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t full0 = cluster_addr(full, 0);  // rank 0's full[0]
      int it = 0;
      bool ok = true;
      for (long long u = cid; u < units && ok; u += ncl) {
        int l, mt, nh, kc;
        unit_coords(u, l, mt, nh, kc);
        const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
        const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          if (it >= S && !mbar_wait_bounded(empty + s, ((it / S) - 1) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * stage_bytes;
          const uint32_t fb = full0 + 8u * static_cast<uint32_t>(s);
          if constexpr (F8) {
            // own staging on own full[s]; rank 0's full[s] also takes both B halves
            mbar_arrive_expect_tx(full + s, static_cast<uint32_t>(kStg + (lead ? 2 * bh_bytes : 0)));
            tma_load_3d(sa + a_bytes + b_all, tmA, kb * BK, mt * kBlockM, l, full + s);
          } else {
            if (lead) mbar_arrive_expect_tx(full + s, 2u * static_cast<uint32_t>(stage_bytes));
            // rows past the last M tile read as zeros (TMA fill); their outputs are never stored
            tma_load_3d_pair(sa, tmA, kb * BK, mt * kBlockM, l, fb);
            if constexpr (SPLIT) tma_load_3d_pair(sa + kA, tmA2, kb * BK, mt * kBlockM, l, fb);
          }
          unsigned char* sb = sa + a_bytes;
          for (int c = 0; c < n_mma; ++c) {
            const int row0 = nh * NU + c * n_mma_cols + static_cast<int>(crank) * hrows;
            tma_load_3d_pair(sb + c * hb, tmB, kb * BK, row0, l, fb);
            if constexpr (SPLIT || BLO) tma_load_3d_pair(sb + bh_bytes + c * hb, tmB2, kb * BK, row0, l, fb);
          }
        }
      }
      if (lead || F8)
        for (int kk = (it > S ? it - S : 0); kk < it; ++kk)
          mbar_wait_bounded(full + kk % S, (kk / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL);
      // the MMAs' releases of the last stages land in both CTAs before anyone leaves
      for (int kk = (it > S ? it - S : 0); kk < it; ++kk)
        mbar_wait_bounded(empty + kk % S, (kk / S) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY);
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      int it = 0, acc_it = 0;
      bool ok = true;
      for (long long u = cid; u < units && ok; u += ncl) {
        int l, mt, nh, kc;
        unit_coords(u, l, mt, nh, kc);
        const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
        const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
        const int as = acc_it % AS;
        if (acc_it >= AS &&
            !mbar_wait_bounded_cl(acc_empty + as, ((acc_it / AS) - 1) & 1, a.status, DEV_ERR_TIMEOUT_MMA)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          const bool got = F8 ? mbar_wait_bounded_cl(aready + s, (it / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL)
                              : mbar_wait_bounded(full + s, (it / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL);
          if (!got) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * stage_bytes);
          const uint32_t sb = sa + a_bytes;
#pragma unroll
          for (int k = 0; k < BK / KI; ++k) {
            const uint64_t ad = sdesc_sw<BKB / 2>(sa + k * 32);
            for (int c = 0; c < n_mma; ++c) {
              const uint32_t boff = c * hb + k * 32;
              const uint64_t bd = sdesc_sw<BKB / 2>(sb + boff);
              const uint32_t dcol = tmem + static_cast<uint32_t>(as * NU + c * n_mma_cols);
              if constexpr (F8F8) {
                tc_mma2_f8f8(dcol, ad, bd, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
                if constexpr (BLO) tc_mma2_f8f8(dcol, ad, sdesc_sw<BKB / 2>(sb + bh_bytes + boff), idesc, 1u);
              } else {
                tc_mma2_bf16(dcol, ad, bd, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
              }
              if constexpr (SPLIT) {
                tc_mma2_bf16(dcol, ad, sdesc_sw<BK>(sb + bh_bytes + boff), idesc, 1u);
                tc_mma2_bf16(dcol, sdesc_sw<BK>(sa + kA + k * 32), bd, idesc, 1u);
              }
            }
          }
          tc_commit2_mc(empty + s, 0x3);
        }
        if (!ok) break;
        tc_commit2_mc(acc_full + as, 0x3);
        ++acc_it;
      }
      // both CTAs' epilogues consume the last accumulators before teardown
      for (int k = (acc_it > AS ? acc_it - AS : 0); k < acc_it; ++k)
        mbar_wait_bounded_cl(acc_empty + k % AS, (k / AS) & 1, a.status, DEV_ERR_TIMEOUT_MMA);
    }
  } else if (F8 && warp >= kConvWarp0) {
    // converter warps of both CTAs: thread t widens row t of this CTA's FP8 A tile
    const int t = threadIdx.x - 32 * kConvWarp0;
    const uint32_t aready0 = cluster_addr(aready, 0);
    int it = 0;
    bool ok = true;
    for (long long u = cid; u < units && ok; u += ncl) {
      int l, mt, nh, kc;
      unit_coords(u, l, mt, nh, kc);
      const int kb0 = a.kb_off + kc * a.kblocks_per_chunk;
      const int kb1 = min(nk_total, kb0 + a.kblocks_per_chunk);
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % S;
        if (!mbar_wait_bounded(full + s, (it / S) & 1, a.status, DEV_ERR_TIMEOUT_FULL)) {
          ok = false;
          break;
        }
        unsigned char* sa = smem + s * stage_bytes;
        widen_fp8_row<BK>(sa + a_bytes + b_all + t * BK, sa + t * (BK * 2), t);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(aready0 + 8u * static_cast<uint32_t>(s));
      }
    }
  } else {
    // epilogue warps of both CTAs: this CTA's 128 rows of the M = 256 tile
    const int q = warp & 3;         // TMEM lane quadrant this warp may access
    const int g = (warp - 2) >> 2;  // column group of the quadrant
    const uint32_t acc_empty0 = cluster_addr(acc_empty, 0);
    int acc_it = 0;
    for (long long u = cid; u < units; u += ncl) {
      int l, mt, nh, kc;
      unit_coords(u, l, mt, nh, kc);
      const int as = acc_it % AS;
      if (!mbar_wait_bounded(acc_full + as, (acc_it / AS) & 1, a.status, DEV_ERR_TIMEOUT_MMA)) break;
      tc_fence_after();
      const int row = mt * kBlockM + q * 32 + lane;
      const uint32_t tbase = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(as * NU);
      const bool live = row < a.M_total && mt < a.m_tiles;
      float scale = 1.f;
      if (a.row_scale != nullptr && live) scale = a.row_scale[static_cast<long long>(l) * a.nblk + row / 256];
      if (a.b_amax != nullptr) scale *= f16_unscale(*a.b_amax);  // undo the FP16 B operand's power-of-two scale
      tc_epilogue_tile<EPW, F8F8>(a, tbase, NU, g, l, kc, row, live, scale,  // F8F8: per-column B scales
                                  F8F8 ? col_scale + static_cast<long long>(l) * col_ld : nullptr, nh * NU / 2);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acc_empty0 + 8u * static_cast<uint32_t>(as));
      ++acc_it;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA still reads or writes the pair's tensor memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc2(tmem, a.tmem_cols);
  }
  cluster_sync_all();  // no CTA leaves while its peer may still signal it
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm2_body<BK, 0>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreadsF8, 1)
    k_tc_gemm2_f8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  tc_gemm2_body<BK, 2>(&tmA, &tmB, nullptr, nullptr, a);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm2_f8f8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a,
                    const float* col_scale, int col_ld) {
  tc_gemm2_body<BK, 3>(&tmA, &tmB, nullptr, nullptr, a, col_scale, col_ld);
}

// FP8 x (hi + lo FP8) MMAs: the slip spectra as two e4m3 parts in one
// power-of-two frame, so the activations keep ~8 bits (as accurate as FP16
// for this use) while both MMAs read 8-bit operands straight from TMA.
template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm2_f8f8lo(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmB2, const TcArgs a, const float* col_scale, int col_ld) {
  tc_gemm2_body<BK, 4>(&tmA, &tmB, nullptr, &tmB2, a, col_scale, col_ld);
}

template <int BK>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm2_split(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                     const TcArgs a) {
  tc_gemm2_body<BK, 1>(&tmA, &tmB, &tmA2, &tmB2, a);
}

// B operand of the real embedding from complex FP32 x[l][t][c] (element
// src[l*s_l + t*s_t + c], c < nc): rows 2t / 2t+1 of dst[l][N_alloc][2 Kc]
// (BF16, round to nearest even) at complex columns c0 + c:
//   plain (D = A x):        row 2t = (Re x, -Im x),  row 2t+1 = (Im x,  Re x)
//   conj  (D = conj(A) x):  row 2t = (Re x,  Im x),  row 2t+1 = (Im x, -Re x)
// With `lo`, lo = bf16(v - hi) holds the low-order part of every entry.
__global__ void k_pack_b(const float2* __restrict__ src, int Nb, int T, long long nc, long long s_l, long long s_t,
                         long long c0, long long Kc, int N_alloc, int conj, __nv_bfloat162* __restrict__ hi,
                         __nv_bfloat162* __restrict__ lo) {
  const long long total = static_cast<long long>(Nb) * T * nc;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = e % nc;
    const long long t = (e / nc) % T;
    const long long l = e / (nc * T);
    const float2 v = src[l * s_l + t * s_t + c];
    if (conj == 2) {  // first half of the plain embedding only: row t = (Re, -Im)
      const long long o = (l * N_alloc + t) * Kc + c0 + c;
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, -v.y);
      hi[o] = h;
      if (lo != nullptr) lo[o] = __floats2bfloat162_rn(v.x - __low2float(h), -v.y - __high2float(h));
      continue;
    }
    const float2 r0 = conj ? make_float2(v.x, v.y) : make_float2(v.x, -v.y);
    const float2 r1 = conj ? make_float2(v.y, -v.x) : make_float2(v.y, v.x);
    const long long o0 = (l * N_alloc + 2 * t) * Kc + c0 + c;
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(r0.x, r0.y);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(r1.x, r1.y);
    hi[o0] = h0;
    hi[o0 + Kc] = h1;
    if (lo != nullptr) {
      lo[o0] = __floats2bfloat162_rn(r0.x - __low2float(h0), r0.y - __high2float(h0));
      lo[o0 + Kc] = __floats2bfloat162_rn(r1.x - __low2float(h1), r1.y - __high2float(h1));
    }
  }
}

// Largest |Re|, |Im| of n complex values into *amax (float bits; *amax
// starts at 0): the range of a B operand packed as FP16.
__global__ void k_amax_c(const float2* __restrict__ x, long long n, unsigned* __restrict__ amax) {
  float m = 0.f;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float2 v = x[e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));  // non-negative floats order as unsigned
}

// As k_pack_b (plain embedding), FP16 entries scaled by f16_scale(*amax).
__global__ void k_pack_b_f16(const float2* __restrict__ src, int Nb, int T, long long nc, long long s_l,
                             long long s_t, long long Kc, int N_alloc, const unsigned* __restrict__ amax,
                             __half2* __restrict__ dst) {
  const float sc = f16_scale(*amax);
  const long long total = static_cast<long long>(Nb) * T * nc;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = e % nc;
    const long long t = (e / nc) % T;
    const long long l = e / (nc * T);
    const float2 v = src[l * s_l + t * s_t + c];
    const long long o0 = (l * N_alloc + 2 * t) * Kc + c;
    dst[o0] = __floats2half2_rn(v.x * sc, -v.y * sc);
    dst[o0 + Kc] = __floats2half2_rn(v.y * sc, v.x * sc);
  }
}

// FP8 B operand: one warp per (bin l, complex column t < n_rows / 2); see
// launch_pack_b_f8.
__global__ void k_pack_b_f8(const float2* __restrict__ src, int Nb, int T, long long nc, long long s_l,
                            long long s_t, long long Kc, int N_alloc, int n_rows, float* __restrict__ col_scale,
                            int col_ld, uint16_t* __restrict__ dst, uint16_t* __restrict__ dst_lo) {
  const int lane = threadIdx.x & 31;
  const int nt = n_rows / 2;
  const long long nw = static_cast<long long>(Nb) * nt;
  for (long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += (static_cast<long long>(gridDim.x) * blockDim.x) >> 5) {
    const long long l = w / nt;
    const int t = static_cast<int>(w % nt);
    uint16_t* r0 = dst + (l * N_alloc + 2 * t) * Kc;  // row 2t: (Re, -Im); row 2t + 1: (Im, Re)
    uint16_t* r1 = r0 + Kc;
    uint16_t* q0 = dst_lo != nullptr ? dst_lo + (l * N_alloc + 2 * t) * Kc : nullptr;
    if (t >= T) {
      for (long long c = lane; c < Kc; c += 32) {
        r0[c] = r1[c] = 0;
        if (q0 != nullptr) q0[c] = q0[Kc + c] = 0;
      }
      if (lane == 0) col_scale[l * col_ld + t] = 0.f;
      continue;
    }
    const float2* x = src + l * s_l + t * s_t;
    float m = 0.f;
    for (long long c = lane; c < nc; c += 32) {
      const float2 v = x[c];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // largest power of two sc with m * sc <= 448 (the exponent of 448 / m)
    float sc = 1.f;
    if (m > 0.f) {
      const float r = fmaxf(fminf(448.f / m, 0x1p100f), 0x1p-100f);
      sc = __uint_as_float(__float_as_uint(r) & 0xff800000u);
    }
    for (long long c = lane; c < Kc; c += 32) {
      const float2 v = c < nc ? x[c] : make_float2(0.f, 0.f);
      const float2 p0 = make_float2(v.x * sc, -v.y * sc), p1 = make_float2(v.y * sc, v.x * sc);
      const __nv_fp8x2_storage_t h0 = __nv_cvt_float2_to_fp8x2(p0, __NV_SATFINITE, __NV_E4M3);
      const __nv_fp8x2_storage_t h1 = __nv_cvt_float2_to_fp8x2(p1, __NV_SATFINITE, __NV_E4M3);
      r0[c] = h0;
      r1[c] = h1;
      if (q0 != nullptr) {  // low-order parts: the rounding remainders, rounded again (same frame)
        const float2 b0 = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h0, __NV_E4M3)));
        const float2 b1 = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h1, __NV_E4M3)));
        q0[c] = __nv_cvt_float2_to_fp8x2(make_float2(p0.x - b0.x, p0.y - b0.y), __NV_SATFINITE, __NV_E4M3);
        q0[Kc + c] = __nv_cvt_float2_to_fp8x2(make_float2(p1.x - b1.x, p1.y - b1.y), __NV_SATFINITE, __NV_E4M3);
      }
    }
    if (lane == 0) col_scale[l * col_ld + t] = 1.f / sc;
  }
}

// A operand (K-major, complex pairs interleaved along K) from complex FP32
// x[l][r][c] (src[l*s_l + r*s_r + c*s_c], r < rows, c < nc):
// dst[(l*rows_total + r0 + r)*Kc + c0 + c] hi (and lo) BF16 pairs.  With
// s_r = 1 and s_c = the source row pitch this is a transposing copy.
__global__ void k_pack_a(const float2* __restrict__ src, int Nb, int rows, long long nc, long long s_l,
                         long long s_r, long long s_c, long long rows_total, long long r0, long long c0, long long Kc,
                         __nv_bfloat162* __restrict__ hi, __nv_bfloat162* __restrict__ lo) {
  const long long total = static_cast<long long>(Nb) * rows * nc;
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = e % nc;
    const long long r = (e / nc) % rows;
    const long long l = e / (nc * rows);
    const float2 v = src[l * s_l + r * s_r + c * s_c];
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const long long o = (l * rows_total + r0 + r) * Kc + c0 + c;
    hi[o] = h;
    if (lo != nullptr) lo[o] = __floats2bfloat162_rn(v.x - __low2float(h), v.y - __high2float(h));
  }
}

// ---------------------------------------------------------------------------
// Retransform as a GEMM (tensor-engine path).  For one signal (grid point i,
// rupture b) the stage-1 -> stage-2 step of the pipeline
//   vhat = FFT( ZeroPad( D_t( Truncate( IFFT(mhat) ) ) ) )
// is a fixed real-linear map of its Nt + 1 bins.  Bins 0 and Nt of a real
// signal are real, so both sides have exactly K = 2 Nt real degrees of
// freedom, ordered  k = 0: Re bin 0,  k = 1: Re bin Nt,  k = 2l, 2l+1:
// Re, Im of bin l (0 < l < Nt).  With T[n][k] (built on the host in FP64 from
// the definitions, rounded to BF16) every tile of 128 signals is
//   V (128 x K) = M (128 x K) T^T,
// one tcgen05 GEMM per tile, A K-major in 128-byte (BF16) or 64-byte
// (split) swizzled k-block slots written by eight fill warps, one k-block
// each so that all of a tile's loads are in flight together (coalesced loads
// of mhat[l][b][i0 .. i0 + 127], 16-byte swizzled stores; split: the FP32
// spectra split into hi + lo on the way).  T streams through a ring by TMA
// (it stays in L2); the accumulator rows go back out as BF16 velocity
// spectra in the stage-2 operand layout.
// Warps: 0 TMA (T), 1 TMEM + MMA, then 4 RT_EPW epilogue warps (RT_EPW per
// TMEM lane quadrant, each taking every RT_EPW-th 64-column chunk of an
// accumulator unit), then the 8 fill warps.  The split kernel keeps one
// epilogue warp per quadrant (its fill warps need the registers).
// ---------------------------------------------------------------------------
constexpr int kRtFillWarps = 8;
__host__ __device__ constexpr int rt_epw(bool split) { return split ? 1 : 2; }
__host__ __device__ constexpr int rt_threads(bool split) { return 32 * (2 + 4 * rt_epw(split) + kRtFillWarps); }

// Schedule.  A tile's K = 2 Nt output columns are at most two 256-column MMA
// halves.  BF16 runs the halves outer: each half is one accumulator unit of
// 256 columns, tensor memory holds two units, and the epilogue drains one
// unit while the MMAs fill the other (a whole 512-column tile would fill
// tensor memory and make the next tile's MMAs wait for its drain).  The M
// tile then stays whole in a ring of RA = 8 k-block slots (K / 64 <= 8) until
// the second half has used it.  Split mode at Nt = 256 cannot hold its
// doubled M tile whole: it runs the K blocks outer and both halves inner in
// one 512-column unit, so each k-block slot is freed once both halves have
// used it.  With a single half (Nt <= 128) both orders coincide and two
// units of K columns fit.
// SPLIT: the FP32 seafloor spectra are split by the fill warps into hi + lo
// BF16 parts, T comes as hi + lo (both from the FP64 matrix), three MMAs per
// K step (hi hi, hi lo, lo hi), and the epilogue writes hi + lo velocity
// spectra (the split stage-2 A operand); 32-element K blocks (64-byte
// swizzle) keep the doubled slots inside shared memory.
// PAIR (BF16 only): two-SM tiles as in tc_gemm2_body.  A cluster of two
// CTAs takes two consecutive 128-signal tiles of one rupture as one M = 256
// tile; each CTA fills its own signals and stages half of every 256-row
// slice of T (rank r: rows r 128 .. of the slice), so the T bytes staged and
// read per CTA halve.  Rank 0 issues the MMAs; both CTAs' fill warps arrive
// on rank 0's afull, both CTAs' T loads complete on rank 0's tfull, and the
// MMA commits arrive on tempty / afree / acc_full of both CTAs (mbarrier
// arrives with a CTA mask; no data moves).
template <bool SPLIT, bool PAIR>
__global__ void __launch_bounds__(rt_threads(SPLIT), 1)
    k_tc_retransform(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmT2,
                     const TcRtArgs a) {
  static_assert(!(SPLIT && PAIR), "two-SM retransform: BF16 only");
  constexpr int BK = SPLIT ? 32 : 64;        // K elements per k-block
  constexpr int EPW = rt_epw(SPLIT);
  constexpr int kFill0 = 2 + 4 * EPW;        // first fill warp
  constexpr int kAs = kBlockM * BK * 2;      // one BF16 part of an M-tile k-block
  constexpr int a_slot = kAs * (SPLIT ? 2 : 1);
  constexpr int kBins = BK / 2;              // complex bins per k-block
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int Nt = a.Nt;
  const int K = 2 * Nt;           // = N
  const int KB = K / BK;          // k-blocks per tile
  const int n_half = K > 256 ? 2 : 1;   // MMA column halves (256 output columns each)
  const int ncols = K > 256 ? 256 : K;
  const bool hout = !SPLIT || n_half == 1;  // halves outer (see the schedule above)
  const int U = hout ? n_half : 1;          // accumulator units per tile
  const int H = hout ? 1 : n_half;          // halves per unit
  const int ucols = H * ncols;              // accumulator columns per unit
  const int AS = 2 * ucols <= 512 ? 2 : 1;  // accumulator units in tensor memory
  const int trows = PAIR ? ncols / 2 : ncols;  // T rows this CTA stages per half
  const int t_part = trows * BK * 2;
  const int t_slot = t_part * (SPLIT ? 2 : 1);
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  const bool lead = crank == 0;
  const long long cid = PAIR ? static_cast<long long>(cluster_id_x()) : static_cast<long long>(blockIdx.x);
  const long long ncl = PAIR ? static_cast<long long>(cluster_count_x()) : static_cast<long long>(gridDim.x);
  // RA k-block slots (>= KB: the BF16 order keeps a whole M tile), one per
  // fill warp: with KB a power of two, slot s = n % RA is only
  // ever filled by one warp (k-blocks kb = s mod KB, or s when KB >= RA), one
  // ring lap apart, so no parity wait can run a phase ahead
  constexpr int RA = kRtFillWarps;
  const int RT = a.rt;
  unsigned char* sA = smem;                  // RA k-block slots
  unsigned char* sT = smem + RA * a_slot;    // RT slots of T
  uint64_t* afull = reinterpret_cast<uint64_t*>(sT + RT * t_slot);
  uint64_t* afree = afull + RA;
  uint64_t* tfull = afree + RA;
  uint64_t* tempty = tfull + RT;
  uint64_t* acc_full = tempty + RT;        // [AS]
  uint64_t* acc_empty = acc_full + 2;      // [AS]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + 2);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int mtiles = (a.Ng + kBlockM - 1) / kBlockM;
  const int mgroups = PAIR ? (mtiles + 1) / 2 : mtiles;  // M tiles per unit: 2 (pair) or 1
  const long long tiles = static_cast<long long>(a.Bs) * mgroups;
  // unit u -> rupture b and this CTA's first signal i0
  auto unit_tile = [&](long long u, int& b, int& i0) {
    b = static_cast<int>(u / mgroups);
    i0 = (static_cast<int>(u % mgroups) * (PAIR ? 2 : 1) + static_cast<int>(crank)) * kBlockM;
  };
  const uint32_t idesc = idesc_bf16(PAIR ? 2 * kBlockM : kBlockM, ncols);
  const int acols = AS * ucols;
  const uint32_t tmem_cols = acols <= 64 ? 64 : (acols <= 128 ? 128 : (acols <= 256 ? 256 : 512));

  if (threadIdx.x == 0) {
    for (int s = 0; s < RA; ++s) {
      mbar_init(afull + s, PAIR ? 2 : 1);  // the k-block's fill warp (of each CTA)
      mbar_init(afree + s, 1);
    }
    for (int s = 0; s < RT; ++s) {
      mbar_init(tfull + s, 1);
      mbar_init(tempty + s, 1);
    }
    for (int s = 0; s < AS; ++s) {
      mbar_init(acc_full + s, 1);
      mbar_init(acc_empty + s, (PAIR ? 2 : 1) * 4 * EPW);
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc2(tmem_holder, tmem_cols);
      tmem_relinquish2();
    } else {
      tmem_alloc(tmem_holder, tmem_cols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();  // both CTAs' barriers and tensor memory exist
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // T slots in job order: tile, unit, k-block, half within the unit
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      const uint32_t tfull0 = PAIR ? cluster_addr(tfull, 0) : 0u;
      for (long long t = cid; t < tiles && ok; t += ncl) {
        for (int u = 0; u < U && ok; ++u) {
          for (int kb = 0; kb < KB && ok; ++kb) {
            for (int hh = 0; hh < H; ++hh, ++it) {
              const int h = hout ? u : hh;
              const int s = it % RT;
              if (it >= RT && !mbar_wait_bounded(tempty + s, ((it / RT) - 1) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY)) {
                ok = false;
                break;
              }
              if constexpr (PAIR) {
                if (lead) mbar_arrive_expect_tx(tfull + s, 2u * static_cast<uint32_t>(t_slot));
                tma_load_3d_pair(sT + s * t_slot, &tmT, kb * BK, h * ncols + static_cast<int>(crank) * trows, 0,
                                 tfull0 + 8u * static_cast<uint32_t>(s));
              } else {
                mbar_arrive_expect_tx(tfull + s, t_slot);
                tma_load_3d(sT + s * t_slot, &tmT, kb * BK, h * ncols, 0, tfull + s);
                if constexpr (SPLIT) tma_load_3d(sT + s * t_slot + t_part, &tmT2, kb * BK, h * ncols, 0, tfull + s);
              }
            }
          }
        }
      }
      if (lead)
        for (int kk = (it > RT ? it - RT : 0); kk < it; ++kk)
          mbar_wait_bounded(tfull + kk % RT, (kk / RT) & 1, a.status, DEV_ERR_TIMEOUT_FULL);
      if constexpr (PAIR)  // the MMAs' releases of the last T slots land in both CTAs before anyone leaves
        for (int kk = (it > RT ? it - RT : 0); kk < it; ++kk)
          mbar_wait_bounded(tempty + kk % RT, (kk / RT) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY);
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // arrivals from the peer CTA (PAIR) need cluster-scope acquire
      auto wait_x = [&](uint64_t* bar, uint32_t parity, int code) {
        return PAIR ? mbar_wait_bounded_cl(bar, parity, a.status, code) : mbar_wait_bounded(bar, parity, a.status, code);
      };
      auto commit = [&](uint64_t* bar) {
        if constexpr (PAIR)
          tc_commit2_mc(bar, 0x3);
        else
          tc_commit(bar);
      };
      int it = 0, tl = 0, un = 0;  // T slot, tile and accumulator unit counters
      bool ok = true;
      for (long long t = cid; t < tiles && ok; t += ncl, ++tl) {
        for (int u = 0; u < U && ok; ++u, ++un) {
          const int as = un % AS;
          if (un >= AS && !wait_x(acc_empty + as, ((un / AS) - 1) & 1, DEV_ERR_TIMEOUT_MMA)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dcol = tmem + static_cast<uint32_t>(as * ucols);
          for (int kb = 0; kb < KB && ok; ++kb) {
            const long long n = static_cast<long long>(tl) * KB + kb;
            const int sa = static_cast<int>(n % RA);
            if (u == 0 && !wait_x(afull + sa, static_cast<int>((n / RA) & 1), DEV_ERR_TIMEOUT_FULL)) {
              ok = false;
              break;
            }
            for (int hh = 0; hh < H; ++hh, ++it) {
              const int s = it % RT;
              if (!mbar_wait_bounded(tfull + s, (it / RT) & 1, a.status, DEV_ERR_TIMEOUT_FULL)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t ua = smem_u32(sA + sa * a_slot);
              const uint32_t ub = smem_u32(sT + s * t_slot);
              const uint32_t d = dcol + static_cast<uint32_t>(hh * ncols);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint64_t ad = sdesc_sw<BK>(ua + k * 32);
                const uint64_t bd = sdesc_sw<BK>(ub + k * 32);
                if constexpr (PAIR)
                  tc_mma2_bf16(d, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                else
                  tc_mma_bf16(d, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                if constexpr (SPLIT) {
                  tc_mma_bf16(d, ad, sdesc_sw<BK>(ub + t_part + k * 32), idesc, 1u);
                  tc_mma_bf16(d, sdesc_sw<BK>(ua + kAs + k * 32), bd, idesc, 1u);
                }
              }
              commit(tempty + s);
            }
            if (!ok) break;
            if (u == U - 1) commit(afree + sa);  // the last unit has used this k-block
          }
          if (!ok) break;
          commit(acc_full + as);
        }
      }
      // the epilogue's releases of the last units (from both CTAs) have landed
      for (int k = (un > AS ? un - AS : 0); k < un; ++k) wait_x(acc_empty + k % AS, (k / AS) & 1, DEV_ERR_TIMEOUT_MMA);
    }
  } else if (warp < kFill0) {
    // epilogue: accumulator row = signal, columns = output degrees of freedom
    const int q = warp & 3;
    const int g = (warp - 2) >> 2;  // column group of the quadrant
    const uint32_t acc_empty0 = PAIR ? cluster_addr(acc_empty, 0) : 0u;
    int un = 0;
    bool ok = true;
    for (long long t = cid; t < tiles && ok; t += ncl) {
      int b, i0;
      unit_tile(t, b, i0);
      const int i = i0 + q * 32 + lane;
      __nv_bfloat162* out = a.vhat + static_cast<long long>(b) * a.vld_b + i;
      __nv_bfloat162* out_lo = SPLIT ? a.vhat_lo + static_cast<long long>(b) * a.vld_b + i : nullptr;
      auto put1 = [&](long long off, float re, float im) {
        const __nv_bfloat162 hi = __floats2bfloat162_rn(re, im);
        out[off] = hi;
        if constexpr (SPLIT) out_lo[off] = __floats2bfloat162_rn(re - __low2float(hi), im - __high2float(hi));
      };
      auto put = [&](long long off, float re, float im) {
        put1(off, re, im);
        if (a.conj_row > 0) put1(off + a.conj_row, im, -re);  // row 2b + 1 of the conjugate embedding
      };
      for (int u = 0; u < U; ++u, ++un) {
        const int as = un % AS;
        if (!mbar_wait_bounded(acc_full + as, (un / AS) & 1, a.status, DEV_ERR_TIMEOUT_MMA)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(as * ucols);
        const int cb = hout ? u * ncols : 0;  // first output column of the unit
        // K = 2 Nt is a multiple of 64 for every supported Nt (32..256)
        for (int c0 = 64 * g; c0 < ucols; c0 += 64 * EPW) {
          float v[64];
          tmem_ld64(tbase + c0, v);
          if (i >= a.Ng) continue;
          const int oc = cb + c0;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int l = oc / 2 + k;
            if (l == 0) {
              put(0, v[0], 0.f);
              put(static_cast<long long>(Nt) * a.vld_l, v[1], 0.f);
            } else {
              put(static_cast<long long>(l) * a.vld_l, v[2 * k], v[2 * k + 1]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(acc_empty0 + 8u * static_cast<uint32_t>(as));
          else
            mbar_arrive(acc_empty + as);
        }
      }
    }
  } else if constexpr (!SPLIT) {
    // fill warps (BF16): warp f fills k-blocks f, f + 8, ... of every tile
    // (k-block kb holds bins 32 kb .. 32 kb + 31 for 128 signals; K slot 1
    // of bin 0 carries Re(bin Nt)), two batches of 16 bins each with 64
    // loads in flight per lane.  The first batch is loaded before the wait
    // for the slot, so its HBM latency overlaps the MMAs that still read the
    // slot; 16-byte chunks are stored in the TMA 128-byte swizzle pattern
    // (chunk ^ (row & 7)).
    const int f = warp - kFill0;
    const uint32_t afull0 = PAIR ? cluster_addr(afull, 0) : 0u;
    int tl = 0;
    bool ok = true;
    for (long long t = cid; t < tiles && ok; t += ncl, ++tl) {
      int b, i0;
      unit_tile(t, b, i0);
      const unsigned* mbb = reinterpret_cast<const unsigned*>(a.mhat_bf) + static_cast<long long>(b) * a.ld_b;
      for (int kb = f; kb < KB && ok; kb += kRtFillWarps) {
        const long long n = static_cast<long long>(tl) * KB + kb;
        const int sa = static_cast<int>(n % RA);
        unsigned raw[16][4];
        auto load = [&](int hh) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long lo = static_cast<long long>(kb * kBins + 16 * hh + j) * a.ld_l;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int i = i0 + 32 * g + lane;
              raw[j][g] = i < a.Ng ? __ldg(mbb + lo + i) : 0u;
            }
          }
        };
        unsigned char* slot = sA + sa * a_slot;
        auto store = [&](int hh) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int row = 32 * g + lane;
              *reinterpret_cast<uint4*>(slot + row * 128 + (((4 * hh + c) ^ (row & 7)) << 4)) =
                  make_uint4(raw[4 * c][g], raw[4 * c + 1][g], raw[4 * c + 2][g], raw[4 * c + 3][g]);
            }
          }
        };
        load(0);
        if (kb == 0) {
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int i = i0 + 32 * g + lane;
            const unsigned rn = i < a.Ng ? __ldg(mbb + static_cast<long long>(Nt) * a.ld_l + i) : 0u;
            raw[0][g] = (raw[0][g] & 0xffffu) | (rn << 16);  // K slot 1: Re(bin Nt)
          }
        }
        if (n >= RA &&
            !mbar_wait_bounded(afree + sa, static_cast<int>(((n / RA) - 1) & 1), a.status, DEV_ERR_TIMEOUT_EMPTY)) {
          ok = false;
          break;
        }
        store(0);
#pragma unroll
        for (int hh = 1; hh < kBins / 16; ++hh) {
          load(hh);
          store(hh);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(afull0 + 8u * static_cast<uint32_t>(sa));
          else
            mbar_arrive(afull + sa);
        }
      }
    }
  } else {
    // fill warps (split): warp f fills k-blocks f, f + 8, ... of every tile
    // (k-block kb holds bins kBins kb .. kBins kb + kBins - 1 for 128 signals;
    // K slot 1 of bin 0 carries Re(bin Nt)); all of a tile's loads are in
    // flight together; 16-byte chunks are stored in the TMA swizzle pattern
    const int f = warp - kFill0;
    int tl = 0;
    bool ok = true;
    for (long long t = cid; t < tiles && ok; t += ncl, ++tl) {
      int b, i0;
      unit_tile(t, b, i0);
      for (int kb = f; kb < KB && ok; kb += kRtFillWarps) {
        const long long n = static_cast<long long>(tl) * KB + kb;
        const int sa = static_cast<int>(n % RA);
        if (n >= RA &&
            !mbar_wait_bounded(afree + sa, static_cast<int>(((n / RA) - 1) & 1), a.status, DEV_ERR_TIMEOUT_EMPTY)) {
          ok = false;
          break;
        }
        unsigned char* slot = sA + sa * a_slot;
        auto chunk_off = [&](int row, int chunk) {  // 16-byte chunk `chunk` of K-major row `row` (64-byte swizzle)
          return row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4);
        };
        const float2* mb = a.mhat32 + static_cast<long long>(b) * a.ld_b;
        float rawn[4] = {0.f, 0.f, 0.f, 0.f};
        if (kb == 0) {
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int i = i0 + 32 * g + lane;
            rawn[g] = i < a.Ng ? __ldg(mb + static_cast<long long>(Nt) * a.ld_l + i).x : 0.f;
          }
        }
#pragma unroll
        for (int hh = 0; hh < kBins / 8; ++hh) {  // 8 bins per batch, 32 float2 loads in flight
          float2 raw[8][4];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long lo = static_cast<long long>(kb * kBins + 8 * hh + j) * a.ld_l;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int i = i0 + 32 * g + lane;
              raw[j][g] = i < a.Ng ? __ldg(mb + lo + i) : make_float2(0.f, 0.f);
            }
          }
          if (kb == 0 && hh == 0) {
#pragma unroll
            for (int g = 0; g < 4; ++g) raw[0][g].y = rawn[g];  // K slot 1: Re(bin Nt)
          }
#pragma unroll
          for (int c = 0; c < 2; ++c) {  // chunk 2 hh + c = bins 8 hh + 4 c .. + 3
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int row = 32 * g + lane;
              unsigned hw[4], lw[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 x = raw[4 * c + e][g];
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(x.x, x.y);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(x.x - __low2float(h2), x.y - __high2float(h2));
                hw[e] = *reinterpret_cast<const unsigned*>(&h2);
                lw[e] = *reinterpret_cast<const unsigned*>(&l2);
              }
              const int off = chunk_off(row, 2 * hh + c);
              *reinterpret_cast<uint4*>(slot + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(slot + kAs + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(afull + sa);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();  // neither CTA still uses the pair's tensor memory
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR)
      tmem_dealloc2(tmem, tmem_cols);
    else
      tmem_dealloc(tmem, tmem_cols);
  }
  if constexpr (PAIR) cluster_sync_all();  // no CTA leaves while its peer may still signal it
}

int grid_for_tc(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 32) g = 152LL * 32;
  return static_cast<int>(g < 1 ? 1 : g);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

namespace {
cudaError_t resolve_encode() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}
}  // namespace

cudaError_t tc_encode_3d(CUtensorMap* out, const void* base, long long K, long long rows, long long nbatch,
                         long long row_pitch_elems, int box_rows, int bk) {
  if (g_encode == nullptr && resolve_encode() != cudaSuccess) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(nbatch)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(row_pitch_elems) * 2,
                                 static_cast<cuuint64_t>(row_pitch_elems) * 2 * static_cast<cuuint64_t>(rows)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_encode_3d_u8(CUtensorMap* out, const void* base, long long K, long long rows, long long nbatch,
                            int box_rows, int bk, int sw128) {
  // sw128 = 1: 128-byte swizzle (bk = 128); 2: 64-byte swizzle (bk = 64)
  if ((sw128 == 1 && bk != 128) || (sw128 == 2 && bk != 64) || sw128 < 0 || sw128 > 2) return cudaErrorInvalidValue;
  if (g_encode == nullptr && resolve_encode() != cudaSuccess) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(nbatch)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(K) * static_cast<cuuint64_t>(rows)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        sw128 == 1 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : (sw128 == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE),
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_block_k(int N, int split, int pair) {
  if (pair) {  // half of B per CTA: 128-byte swizzle whenever four such stages fit
    const int stage64 = (kBlockM + N / 2) * 64 * 2 * (1 + split);
    return 4 * stage64 <= kSmemBudget ? 64 : 32;
  }
  return (N > 256 || (split && N > 128)) ? 32 : 64;
}

namespace {
int tc_stage_bytes(int N, int a_lo, int b_lo, int fp8, int mt) {
  const int bk = tc_block_k(N, a_lo | b_lo);
  return kBlockM * bk * 2 * (1 + a_lo) * mt + N * bk * 2 * (1 + b_lo) + (fp8 ? kBlockM * bk : 0);
}
}  // namespace

int tc_stages_for(int N, int a_lo, int b_lo, int fp8, int mt) {
  // (a fifth FP8 stage at N = 512 from the opt-in shared memory measured no gain)
  int s = kSmemBudget / tc_stage_bytes(N, a_lo, b_lo, fp8, mt);
  if (s > 8) s = 8;
  return s;
}

size_t tc_smem_bytes(int N, int stages, int a_lo, int b_lo, int fp8, int mt) {
  return 1024 + static_cast<size_t>(stages) * tc_stage_bytes(N, a_lo, b_lo, fp8, mt) + 8 * (3 * stages + 2) + 16;
}

namespace {
// Two-SM form: per CTA, one A tile and half of the B tile (each part
// doubled when split), plus the byte staging of an FP8 A tile.  N: the
// columns of one unit (N / 2 with n_split = 2).
// fp8 = 2: FP8 A and B read directly (128-byte rows of 128 K elements);
// fp8 = 3: the same with B as hi + lo parts (64-byte rows of 64 K elements);
// fp8 = 4: hi + lo B parts in 128-byte rows of 128 K elements (n_split).
int tc2_stage_bytes(int N, int split, int fp8) {
  if (fp8 == 2) return (kBlockM + N / 2) * 128;
  if (fp8 == 3) return (kBlockM + N) * 64;
  if (fp8 == 4) return (kBlockM + N) * 128;
  const int bk = tc_block_k(N, split, 1);
  return (kBlockM * bk * 2 + (N / 2) * bk * 2) * (1 + split) + (fp8 ? kBlockM * bk : 0);
}
size_t tc2_smem_bytes(int N, int stages, int split, int fp8) {
  return 1024 + static_cast<size_t>(stages) * tc2_stage_bytes(N, split, fp8) + 8 * (3 * stages + 2) + 16;
}
constexpr int kSmemOptIn = 227 * 1024;
}  // namespace

int tc_stages_pair(int N, int split, int fp8) {
  // FP8 stages that carry the staging too may use all of the opt-in shared
  // memory (four 56 KB stages at N = 512)
  const int budget = fp8 == 1 ? kSmemOptIn - 1024 - 8 * (3 * 8 + 2) - 16 : kSmemBudget;
  int s = budget / tc2_stage_bytes(N, split, fp8);
  if (s > 8) s = 8;
  return s;
}

// One CTA per SM (persistent over the units), one CTA per 128-row tile.
template <int BK, int MODE>
cudaError_t launch_tc_one(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmA2,
                          const CUtensorMap& tmB2, const TcArgs& a, int num_sms, size_t smem, cudaStream_t st) {
  auto kern = k_tc_gemm<BK>;
  auto kern_s = k_tc_gemm_split<BK>;
  auto kern_f = k_tc_gemm_f8<BK>;
  const void* kfn = MODE == 1   ? reinterpret_cast<const void*>(kern_s)
                    : MODE == 2 ? reinterpret_cast<const void*>(kern_f)
                                : reinterpret_cast<const void*>(kern);
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long units = static_cast<long long>(a.Nb) * a.m_tiles * a.n_kchunks;
  const unsigned grid = static_cast<unsigned>(units < num_sms ? units : num_sms);
  const unsigned threads = MODE == 2 ? kTcThreadsF8 : kTcThreads;
  if (MODE == 1)
    kern_s<<<grid, threads, smem, st>>>(tmA, tmB, tmA2, tmB2, a);
  else if (MODE == 2)
    kern_f<<<grid, threads, smem, st>>>(tmA, tmB, a);
  else
    kern<<<grid, threads, smem, st>>>(tmA, tmB, a);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcArgs& a, int num_sms,
                           cudaStream_t st, const CUtensorMap* tmA2, const CUtensorMap* tmB2, const float* col_scale,
                           int col_ld) {
  const long long units = static_cast<long long>(a.Nb) * a.m_tiles * a.n_kchunks;
  if (units <= 0) return cudaSuccess;
  if (a.N < 16 || a.N > 512 || a.N % 16 != 0 || (a.N > 256 && a.N % 256 != 0) || a.stages < 2)
    return cudaErrorInvalidValue;
  // split operands come in pairs: both A and B carry lo parts, or neither;
  // FP8 A (a_fp8) takes a byte tensor map and excludes the split
  if (a.a_lo != a.b_lo || (a.a_lo != 0 && a.a_lo != 1) || (a.a_lo && (!tmA2 || !tmB2))) return cudaErrorInvalidValue;
  if ((a.a_fp8 != 0 && a.a_fp8 != 1) || (a.a_fp8 && a.a_lo) || (a.a_fp8 && a.row_scale == nullptr))
    return cudaErrorInvalidValue;
  if (a.b_half) {  // B as its first N / 2 rows; the converter warps build the rest
    if (a.cta2 || a.a_lo || a.b_lo || a.a_fp8 || col_scale != nullptr || a.N > 256 || a.N % 32 != 0 ||
        tc_block_k(a.N, 0) != 64)
      return cudaErrorInvalidValue;
    const int mt = a.m_pair ? 2 : 1;
    const size_t smem = tc_smem_bytes(a.N, a.stages, 0, 0, 0, mt);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const long long pu = static_cast<long long>(a.Nb) * ((a.m_tiles + mt - 1) / mt) * a.n_kchunks;
    const unsigned grid = static_cast<unsigned>(pu < num_sms ? pu : num_sms);
    const void* kfn = a.m_pair ? reinterpret_cast<const void*>(k_tc_gemm_pair_h<64>)
                               : reinterpret_cast<const void*>(k_tc_gemm_h<64>);
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (a.m_pair)
      k_tc_gemm_pair_h<64><<<grid, kTcThreadsF8, smem, st>>>(tmA, tmB, a);
    else
      k_tc_gemm_h<64><<<grid, kTcThreadsF8, smem, st>>>(tmA, tmB, a);
    return cudaGetLastError();
  }
  if (a.cta2) {  // two-SM MMAs (M = 256 per CTA pair), no M-tile pairs
    if (a.m_pair || a.N % 32 != 0) return cudaErrorInvalidValue;
    const int sp = a.a_lo;
    const int f8 = a.a_fp8;
    const bool f8f8 = col_scale != nullptr;
    const bool f8lo = f8f8 && tmB2 != nullptr;  // B as hi + lo e4m3 parts
    if (f8f8 && (!a.a_fp8 || col_ld < a.T)) return cudaErrorInvalidValue;
    const bool nsp = a.n_split == 2;  // FP8 x (hi + lo FP8) at N = 512 only
    if ((a.n_split != 0 && a.n_split != 1 && !nsp) || (nsp && (!f8lo || a.N != 512))) return cudaErrorInvalidValue;
    const size_t smem =
        tc2_smem_bytes(nsp ? a.N / 2 : a.N, a.stages, sp, f8lo ? (nsp ? 4 : 3) : (f8f8 ? 2 : f8));
    if (smem > static_cast<size_t>(kSmemOptIn)) return cudaErrorInvalidValue;
    const bool bk64 = tc_block_k(a.N, sp, 1) == 64;
    const void* kfn = f8lo ? (nsp ? reinterpret_cast<const void*>(k_tc_gemm2_f8f8lo<128>)
                                  : reinterpret_cast<const void*>(k_tc_gemm2_f8f8lo<64>))
                      : f8f8 ? reinterpret_cast<const void*>(k_tc_gemm2_f8f8<128>)
                      : f8 ? (bk64 ? reinterpret_cast<const void*>(k_tc_gemm2_f8<64>)
                                   : reinterpret_cast<const void*>(k_tc_gemm2_f8<32>))
                      : sp ? (bk64 ? reinterpret_cast<const void*>(k_tc_gemm2_split<64>)
                                   : reinterpret_cast<const void*>(k_tc_gemm2_split<32>))
                           : (bk64 ? reinterpret_cast<const void*>(k_tc_gemm2<64>)
                                   : reinterpret_cast<const void*>(k_tc_gemm2<32>));
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(f8 && !f8f8 ? kTcThreadsF8 : kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.gridDim = dim3(static_cast<unsigned>((num_sms / 2) * 2));
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, kfn, &cfg);
    if (e != cudaSuccess) return e;
    if (active < 1) return cudaErrorInvalidConfiguration;
    long long nclusters = active;
    const long long pu = static_cast<long long>(a.Nb) * ((a.m_tiles + 1) / 2) * a.n_kchunks * (nsp ? 2 : 1);
    if (nclusters > pu) nclusters = pu;
    cfg.gridDim = dim3(static_cast<unsigned>(nclusters * 2));
    if (f8lo) {
      if (nsp)
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_f8f8lo<128>, tmA, tmB, *tmB2, a, col_scale, col_ld);
      else
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_f8f8lo<64>, tmA, tmB, *tmB2, a, col_scale, col_ld);
    } else if (f8f8) {
      e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_f8f8<128>, tmA, tmB, a, col_scale, col_ld);
    } else if (f8) {
      if (bk64)
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_f8<64>, tmA, tmB, a);
      else
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_f8<32>, tmA, tmB, a);
    } else if (sp) {
      if (bk64)
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_split<64>, tmA, tmB, *tmA2, *tmB2, a);
      else
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2_split<32>, tmA, tmB, *tmA2, *tmB2, a);
    } else {
      if (bk64)
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2<64>, tmA, tmB, a);
      else
        e = cudaLaunchKernelEx(&cfg, k_tc_gemm2<32>, tmA, tmB, a);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  if (col_scale != nullptr) return cudaErrorInvalidValue;  // FP8 B: two-SM form only
  const int mt = a.m_pair ? 2 : 1;
  if (a.m_pair && (a.N > 256 || a.a_fp8)) return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes(a.N, a.stages, a.a_lo, a.b_lo, a.a_fp8, mt);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (a.m_pair) {  // pairs of M tiles per unit
    const long long pu = static_cast<long long>(a.Nb) * ((a.m_tiles + 1) / 2) * a.n_kchunks;
    const unsigned grid = static_cast<unsigned>(pu < num_sms ? pu : num_sms);
    const bool bk64 = tc_block_k(a.N, a.a_lo) == 64;
    const void* kfn = a.a_lo ? (bk64 ? reinterpret_cast<const void*>(k_tc_gemm_split_pair<64>)
                                     : reinterpret_cast<const void*>(k_tc_gemm_split_pair<32>))
                             : (bk64 ? reinterpret_cast<const void*>(k_tc_gemm_pair<64>)
                                     : reinterpret_cast<const void*>(k_tc_gemm_pair<32>));
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (a.a_lo) {
      if (bk64)
        k_tc_gemm_split_pair<64><<<grid, kTcThreads, smem, st>>>(tmA, tmB, *tmA2, *tmB2, a);
      else
        k_tc_gemm_split_pair<32><<<grid, kTcThreads, smem, st>>>(tmA, tmB, *tmA2, *tmB2, a);
    } else {
      if (bk64)
        k_tc_gemm_pair<64><<<grid, kTcThreads, smem, st>>>(tmA, tmB, a);
      else
        k_tc_gemm_pair<32><<<grid, kTcThreads, smem, st>>>(tmA, tmB, a);
    }
    return cudaGetLastError();
  }
  const CUtensorMap& a2 = a.a_lo ? *tmA2 : tmA;  // unused unless a_lo / b_lo
  const CUtensorMap& b2 = a.b_lo ? *tmB2 : tmB;
  auto go = [&](auto bk_tag, auto mode_tag) -> cudaError_t {
    constexpr int BK = decltype(bk_tag)::value;
    constexpr int MD = decltype(mode_tag)::value;
    return launch_tc_one<BK, MD>(tmA, tmB, a2, b2, a, num_sms, smem, st);
  };
  using bk64 = std::integral_constant<int, 64>;
  using bk32 = std::integral_constant<int, 32>;
  using m0 = std::integral_constant<int, 0>;
  using m1 = std::integral_constant<int, 1>;
  using m2 = std::integral_constant<int, 2>;
  const int mode = a.a_lo ? 1 : (a.a_fp8 ? 2 : 0);
  if (tc_block_k(a.N, mode == 1 ? 1 : 0) == 64) {
    if (mode == 1) return go(bk64{}, m1{});
    return mode == 2 ? go(bk64{}, m2{}) : go(bk64{}, m0{});
  }
  if (mode == 1) return go(bk32{}, m1{});
  return mode == 2 ? go(bk32{}, m2{}) : go(bk32{}, m0{});
}

cudaError_t launch_tc_retransform(const CUtensorMap& tmT, const CUtensorMap* tmT2, const TcRtArgs& a, int num_sms,
                                  cudaStream_t st, const CUtensorMap* tmTp) {
  if (a.Nt < 32 || a.Nt > 256 || a.Nt % 32 != 0) return cudaErrorInvalidValue;
  const int mtiles = (a.Ng + kBlockM - 1) / kBlockM;
  const long long tiles = static_cast<long long>(a.Bs) * mtiles;
  if (tiles <= 0) return cudaSuccess;
  const bool split = tmT2 != nullptr;
  if (split ? (a.mhat32 == nullptr || a.vhat_lo == nullptr) : (a.mhat_bf == nullptr)) return cudaErrorInvalidValue;
  // two-SM tiles (BF16 only) when a half-row map of T is given and the grid spans two M tiles
  const bool pair = !split && tmTp != nullptr && mtiles >= 2;
  const int BK = split ? 32 : 64;
  const int K = 2 * a.Nt;
  const int ncols = K > 256 ? 256 : K;
  const size_t a_slot = static_cast<size_t>(kBlockM) * BK * 2 * (split ? 2 : 1);
  const size_t t_slot = static_cast<size_t>(pair ? ncols / 2 : ncols) * BK * 2 * (split ? 2 : 1);
  TcRtArgs aa = a;
  aa.ra = kRtFillWarps;  // k-block slots of A: a whole tile (BF16), one per fill warp (split)
  // T slots fill the opt-in shared memory left by the A ring (up to four)
  aa.rt = static_cast<int>((kSmemOptInLimit - 1024 - (8 * (2 * aa.ra + 2 * 4 + 4) + 16) - aa.ra * a_slot) / t_slot);
  if (aa.rt > 4) aa.rt = 4;
  if (aa.rt < 2) return cudaErrorInvalidValue;
  const size_t smem = 1024 + aa.ra * a_slot + aa.rt * t_slot + 8 * (2 * aa.ra + 2 * aa.rt + 4) + 16;
  if (pair) {
    const void* kfn = reinterpret_cast<const void*>(k_tc_retransform<false, true>);
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(rt_threads(false));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.gridDim = dim3(static_cast<unsigned>((num_sms / 2) * 2));
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, kfn, &cfg);
    if (e != cudaSuccess) return e;
    if (active < 1) return cudaErrorInvalidConfiguration;
    long long nclusters = active;
    const long long units = static_cast<long long>(a.Bs) * ((mtiles + 1) / 2);
    if (nclusters > units) nclusters = units;
    cfg.gridDim = dim3(static_cast<unsigned>(nclusters * 2));
    e = cudaLaunchKernelEx(&cfg, k_tc_retransform<false, true>, *tmTp, *tmTp, aa);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const long long grid = tiles < num_sms ? tiles : num_sms;
  const void* kfn = split ? reinterpret_cast<const void*>(k_tc_retransform<true, false>)
                          : reinterpret_cast<const void*>(k_tc_retransform<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (split)
    k_tc_retransform<true, false><<<static_cast<unsigned>(grid), rt_threads(true), smem, st>>>(tmT, *tmT2, aa);
  else
    k_tc_retransform<false, false><<<static_cast<unsigned>(grid), rt_threads(false), smem, st>>>(tmT, tmT, aa);
  return cudaGetLastError();
}

cudaError_t launch_pack_b(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t, long long c0,
                          long long Kc, int N_alloc, int conj, void* hi, void* lo, cudaStream_t st) {
  const long long total = static_cast<long long>(Nb) * T * nc;
  if (total <= 0) return cudaSuccess;
  k_pack_b<<<grid_for_tc(total), 256, 0, st>>>(src, Nb, T, nc, s_l, s_t, c0, Kc, N_alloc, conj,
                                               static_cast<__nv_bfloat162*>(hi), static_cast<__nv_bfloat162*>(lo));
  return cudaGetLastError();
}

cudaError_t launch_pack_b_f8(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t,
                             long long Kc, int N_alloc, int n_rows, float* col_scale, int col_ld, void* dst, void* dst_lo,
                             cudaStream_t st) {
  if (n_rows % 2 != 0 || n_rows > N_alloc || 2 * T > n_rows || nc > Kc || col_ld < n_rows / 2)
    return cudaErrorInvalidValue;
  const long long warps = static_cast<long long>(Nb) * (n_rows / 2);
  if (warps <= 0) return cudaSuccess;
  long long blocks = (warps + 7) / 8;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_pack_b_f8<<<static_cast<unsigned>(blocks), 256, 0, st>>>(src, Nb, T, nc, s_l, s_t, Kc, N_alloc, n_rows,
                                                                col_scale, col_ld, static_cast<uint16_t*>(dst),
                                                                static_cast<uint16_t*>(dst_lo));
  return cudaGetLastError();
}

cudaError_t launch_pack_b_f16(const float2* src, int Nb, int T, long long nc, long long s_l, long long s_t,
                              long long Kc, int N_alloc, unsigned* amax, void* dst, cudaStream_t st) {
  const long long total = static_cast<long long>(Nb) * T * nc;
  if (total <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_amax_c<<<grid_for_tc(total), 256, 0, st>>>(src, total, amax);
  k_pack_b_f16<<<grid_for_tc(total), 256, 0, st>>>(src, Nb, T, nc, s_l, s_t, Kc, N_alloc, amax,
                                                   static_cast<__half2*>(dst));
  return cudaGetLastError();
}

cudaError_t launch_pack_a(const float2* src, int Nb, int rows, long long nc, long long s_l, long long s_r,
                          long long s_c, long long rows_total, long long r0, long long c0, long long Kc, void* hi,
                          void* lo, cudaStream_t st) {
  const long long total = static_cast<long long>(Nb) * rows * nc;
  if (total <= 0) return cudaSuccess;
  k_pack_a<<<grid_for_tc(total), 256, 0, st>>>(src, Nb, rows, nc, s_l, s_r, s_c, rows_total, r0, c0, Kc,
                                               static_cast<__nv_bfloat162*>(hi), static_cast<__nv_bfloat162*>(lo));
  return cudaGetLastError();
}

}  // namespace s2w
