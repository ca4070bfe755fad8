// C ABI of libs2w (include/s2w.h): context, operator loading, and the
// waveform pipeline q = F_q D_t F_G s on one GPU.
//
// Pipeline of one s2w_waveforms call (Alg. 1 steps 2-4, each matvec by
// Alg. 2):
//   K1  rfft of every slip row, zero-padded to 2 Nt      -> shat [l][b][Ns_pad]
//   per rupture b:
//     K2  stage-1 per-bin contraction (HBM stream of Ghat) -> mhat [l][Ng]
//     K3  IFFT + Truncate, D_t, ZeroPad + FFT              -> vhat [l][nseg*RL]
//     K4  stage-2 per-bin contraction over grid segments   -> partial [b][l][seg][o]
//   K5  sum of segment partials (the in-device ReduceSum of Alg. 1 step 5)
//       fused with IFFT + Truncate                        -> q [b][o][Nt]
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "s2w_internal.cuh"

using namespace s2w;

struct s2w_ctx {
  int Ns, Ng, No, Nt, Nb, L, Ns_pad;
  int RL, nseg;  // stage-2 grid segments: nseg segments of RL columns
  s2w_opts opts;
  int device, num_sms;
  // resident operators
  void* G = nullptr;
  void* G_lo = nullptr;
  float* G_scale = nullptr;
  int nblk = 0;
  void* P = nullptr;
  void* P_lo = nullptr;   // FP32_HILO: low-order parts of Phat
  size_t g_bytes = 0, p_bytes = 0;
  float2* tw = nullptr;
  // FP32_HILO (FP32 pairs everywhere on the stream path): pair twiddles and
  // the low-order parts of every intermediate spectrum
  bool df = false;
  float4* tw_df = nullptr;
  float2* ws_shat_lo = nullptr;
  float2* ws_mhat_lo = nullptr;
  float2* ws_vhat_lo = nullptr;
  float2* ws_part_lo = nullptr;
  // workspaces
  float* ws_slip = nullptr;
  float2* ws_shat = nullptr;
  float2* ws_mhat = nullptr;
  float2* ws_vhat = nullptr;
  float2* ws_part = nullptr;
  float* ws_q = nullptr;
  float* ws_seafloor = nullptr;
  float2* ws_rhat = nullptr;   // adjoint: residual spectra [l][b][No]
  float* ws_resid = nullptr;   // misfit gradient: q then r = q - d, [b][No][Nt]
  float* ws_d = nullptr;       // misfit gradient: staged targets, [b][No][Nt]
  float* ws_loss = nullptr;    // misfit gradient: per-rupture loss
  float2* ws_gpart = nullptr;  // adjoint: stage-1 chunk partials [l][chunk][Ns_pad]
  int adj_rc = 512;            // adjoint: grid rows per stage-1 chunk
  int adj_nchunk = 1;
  int* d_status = nullptr;
  // tensor-core engine (BF16 storage, rupture batches)
  bool tc_on = false;
  int tc_bsub = 0;       // sub-batch per tensor pass (<= tc_bsub_max)
  int tc_bsub_max = 0;   // sub-batch the tensor workspaces are sized for (<= 256)
  int tc_n1max = 0;      // B-operand rows of stage 1 (2 x sub-batch, padded)
  int tc_n2 = 0;         // B-operand rows of stage 2 (2 x No, padded)
  bool tc_p2h = false;   // stage-2 operand stored as rows (Re, -Im) only (TcArgs::b_half): tc_n2 / 2 rows
  long long Ng_pad2 = 0; // complex columns per row of the stage-2 operands
  int tc_kbpc = 64;      // K blocks per stage-2 chunk
  int tc_nkc = 1;        // stage-2 K chunks (<= s2_max_chunks, the partials' allocation)
  int s2_min_chunks = 1;  // fewest stage-2 chunks the default and the autotuner take (split: kSplitChunkK)
  int s2_max_chunks = 0;  // stage-2 chunks the partials are sized for
  int tc_pair = 0;       // 1: two-SM MMAs (CTA pairs per M = 256 tile) where the shape allows; kPairAuto: for N = 512
  bool tc_rtpair = false;  // two-SM tiles for the BF16 retransform GEMM
  int tc_min_batch = 2;  // AUTO: smallest B on the tensor engine
  // test hooks (s2w_opts.fault): what to inject, and the kernel wait bound
  int fault = S2W_FAULT_NONE;
  unsigned long long wait_ns = kWaitLimitNs;
  std::string tune_cache;  // autotuner cache file (empty: none)
  // CUDA graphs of the waveform pipeline, one per (slip, q, B), least
  // recently used evicted beyond kGraphCache entries
  struct GraphEntry {
    const float* slip;
    float* q;
    int B;
    cudaGraphExec_t exec;
    long long launches;
    unsigned long long last_use;
  };
  cudaStream_t cap_stream = nullptr;
  // host-buffer calls on the tensor engine: copies of one sub-batch overlap
  // the GEMMs of another (copy stream, one event pair per sub-batch)
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_out;
  std::vector<GraphEntry> graphs;
  unsigned long long graph_clock = 0;
  // tensor-engine adjoint: transposed spectra, K-major along the grid
  bool tc_adj = false;
  int NoP = 0;                // complex columns per row of Phat^T (No padded to 32)
  void* tc_gT = nullptr;      // [Nb][Ns][Ng_pad2] bf16 pairs: Ghat_l^T
  void* tc_gT_lo = nullptr;
  void* tc_pT = nullptr;      // [Nb][Ng][NoP] bf16 pairs: Phat_l^T
  void* tc_pT_lo = nullptr;
  void* tc_rb = nullptr;      // [Nb][tc_n1max][2 NoP] bf16: residual spectra, conjugate embedding
  void* tc_rb_lo = nullptr;
  void* tc_ub = nullptr;      // [Nb][tc_n1max][2 Ng_pad2] bf16: D_t^T-retransformed spectra, conjugate embedding
  void* tc_ub_lo = nullptr;
  float2* tc_ghat = nullptr;  // [Nb][tc_bsub][Ns] complex FP32
  bool single_pass = false;     // L = 4 Nt, D_t folded into Phat, no retransform
  int* ws_lens = nullptr;       // active samples per rupture (s2w_waveforms_active), [max_batch]
  unsigned* d_amax = nullptr;   // FP16 B operand of the FP8 tensor path: its amax (float bits)
  const int* cur_lens = nullptr;  // set for the duration of an s2w_waveforms_active call
  bool tc_split = false;    // BF16 hi/lo operands and activations (three MMAs per K step)
  void* tc_bp1_lo = nullptr;  // split: low-order parts of tc_bp1, tc_vhat, tc_p2
  void* tc_vhat_lo = nullptr;
  void* tc_p2_lo = nullptr;
  void* tc_bp1 = nullptr;   // [Nb][tc_n1max][2 Ns_pad] bf16 (FP8 activations: bytes)
  bool tc_f8act = false;    // FP8 operator x FP8 activations on stage 1 (opts.tc_fp8_act 1 or 2)
  bool tc_f8lo = false;     // ... with the activations as hi + lo e4m3 parts (opts.tc_fp8_act = 2)
  float* tc_colscale = nullptr;  // [Nb][tc_n1max / 2] per-(bin, rupture) scales of the FP8 B operand
  void* tc_mhat = nullptr;  // BF16: [Nb][b][Ng_pad2] (Re, Im) pairs; split (and the adjoint): [Nb][b][Ng] complex FP32
  void* tc_vhat = nullptr;  // [Nb][tc_bsub][Ng_pad2] bf16 pairs
  float2* tc_part = nullptr;  // [Nb][nkc][b][No] complex FP32
  void* tc_p2 = nullptr;    // [Nb][tc_n2 (tc_n2 / 2 when tc_p2h)][Ng_pad2] bf16 pairs
  void* tc_T = nullptr;     // [2 Nt][2 Nt] bf16: retransform as a real-linear map
  void* tc_T_lo = nullptr;  // split: its low-order part
  CUtensorMap tc_tmT, tc_tmT2;
  CUtensorMap tc_tmTp, tc_tmTap;  // BF16: the same matrices with half-row boxes (two-SM retransform)
  void* tc_Ta = nullptr;    // tc_adjoint: the same map with D_t^T (adjoint retransform), + lo when split
  void* tc_Ta_lo = nullptr;
  CUtensorMap tc_tmTa, tc_tmTa2;
  std::vector<unsigned char> g_loaded, p_loaded;
  long long g_count = 0, p_count = 0;
  // per-stage event timers
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  double prof_ms[S2W_NUM_STAGES] = {0};
  long long prof_cnt[S2W_NUM_STAGES] = {0};
  long long launches = 0;
  char err[512] = {0};
};

namespace {

thread_local char g_create_err[512];

int fail(s2w_ctx* c, int code, const char* fmt, ...) {
  char* dst = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? S2W_ERR_OOM : S2W_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) return e;
  return cudaMemset(*p, 0, bytes);
}

// 1 = device memory of `device`, 0 = host memory, -1 = device memory of
// another device.
int pointer_kind(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return at.device == device ? 1 : -1;
  return 0;
}

// Tensor engine: whether GEMMs take the two-SM form by default (kPairAuto: for N = 512, where half
// of B per CTA lets the ring take 64-element K blocks with 128-byte swizzle;
// measured 0.86 against 0.75 of the sustained BF16 peak for the 256-rupture
// stage 1.  At N = 128 the M-tile pairs of one CTA were faster, and so
// were single CTAs for FP8 A: 0.63 against 0.50, the pair's cross-CTA
// converter handshake sitting on every stage.)
constexpr int kPairAuto = 2;
constexpr int kDefaultPair = kPairAuto;
// Largest stage-2 split-K chunk count (the tensor partials are sized for it,
// so s2w_autotune and opts.tc_s2_chunks can pick any count up to it).
constexpr int kMaxS2Chunks = 16;
// The split precision's stage-2 chunks hold at most this many K elements by
// default: each chunk is one FP32 accumulation in tensor memory, and at the
// split's error level the length of that accumulation shows (963 x 60,000 x
// 64 x 256, 256 ruptures: one chunk of 120,000 K elements 9.9e-5 rel-L2,
// seven 2.0e-5, against 5.2e-6 from the rounding of the split operands
// alone).  Its partials are sized for the chunk count this takes.
constexpr long long kSplitChunkK = 2048;
// The tensor adjoint's last GEMM (K = the grid) at the split precision runs
// in launches of at most this many K elements, each adding its FP32 partial
// into the output: longer accumulations than stage 2's chunks (each launch
// re-reads and rewrites the output, so fewer of them), short enough for the
// split's error level (963 x 40,000, rel-L2 of the adjoint: one accumulation
// ~2e-4; launches of 8,192 elements 2.9e-5 at +4 % gradient time, of 4,096
// 1.6e-5 at +9 %, of 2,048 9.8e-6 at +21 %).
constexpr long long kSplitAdjChunkK = 4096;

// Form of one tensor GEMM; sets the ring depth and TMEM columns of `a` and
// returns the B tensor map's box rows.  With `pair` (1, or kPairAuto and
// the shape it covers; and N % 32 == 0, at least two M tiles): two-SM MMAs,
// a CTA pair per M = 256 tile staging half of B each.  Otherwise two M tiles
// per unit sharing each B tile when the accumulators fit (N <= 256), for
// non-FP8 A and at least two M tiles.  Every CTA loads its own tiles.
int tc_shape(TcArgs& a, int N, int m_tiles, int split, int fp8, int pair) {
  if (pair == kPairAuto) pair = N == 512 && !split && !fp8;
  a.cta2 = (pair && N % 32 == 0 && m_tiles >= 2) ? 1 : 0;
  a.m_pair = (!a.cta2 && N <= 256 && !fp8 && m_tiles >= 2) ? 1 : 0;
  const int mt = a.m_pair ? 2 : 1;
  a.stages = a.cta2 ? tc_stages_pair(N, split, fp8) : tc_stages_for(N, split, split, fp8, mt);
  const int cols = mt * N;
  a.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
  const int slice = N > 256 ? 256 : N;
  return a.cta2 ? slice / 2 : slice;
}

// Stage-2 split-K over the grid: the chunk count `want` (1..s2_max_chunks), or
// for want = 0 the count from s2_min_chunks up that minimises rounds x chunk
// length over the persistent CTAs for units = bins x M-tile groups (pairs of
// 128-row tiles when the GEMM takes them) x K chunks, with a small fixed cost
// per unit (pipeline fill and accumulator drain).  Sets tc_kbpc and tc_nkc.
void set_s2_chunks(s2w_ctx* ctx, int want) {
  const int bk2 = tc_block_k(ctx->tc_n2, ctx->tc_split ? 1 : 0);
  const long long nk2 = (2 * ctx->Ng_pad2 + bk2 - 1) / bk2;
  const long long cmax = std::min<long long>(ctx->s2_max_chunks, nk2);
  long long nkc = want;
  if (nkc <= 0) {
    const long long mt2 = (ctx->tc_bsub + 127) / 128;
    const long long mg2 = (mt2 >= 2 && ctx->tc_n2 <= 256) ? (mt2 + 1) / 2 : mt2;
    double best = 1e300;
    nkc = 1;
    for (long long c = std::min<long long>(ctx->s2_min_chunks, cmax); c <= cmax; ++c) {
      const long long units = ctx->Nb * mg2 * c;
      const long long rounds = (units + ctx->num_sms - 1) / ctx->num_sms;
      const double cost = static_cast<double>(rounds) * (1.0 / static_cast<double>(c) + 0.005);
      if (cost < best * (1.0 - 1e-9)) {
        best = cost;
        nkc = c;
      }
    }
  }
  nkc = std::max<long long>(1, std::min<long long>(nkc, cmax));
  ctx->tc_kbpc = static_cast<int>((nk2 + nkc - 1) / nkc);
  ctx->tc_nkc = static_cast<int>((nk2 + ctx->tc_kbpc - 1) / ctx->tc_kbpc);
}

// The stream engine handles ruptures in groups of at most this many (its
// per-call workspaces are sized for one group).
constexpr int kStreamGroup = 64;

bool supported_nt(int Nt) { return Nt == 32 || Nt == 64 || Nt == 128 || Nt == 256 || Nt == 512; }

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

cudaEvent_t take_event(s2w_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Brackets one stage launch with CUDA events on its stream when the profiler
// is on; counts `n` kernel launches either way.
struct StageTimer {
  s2w_ctx* c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  StageTimer(s2w_ctx* c_, int stage_, cudaStream_t st_, int n = 1) : c(c_), stage(stage_), st(st_) {
    c->launches += n;
    if (c->prof_on) {
      a = take_event(c);
      b = take_event(c);
      if (a && b) cudaEventRecord(a, st);
    }
  }
  ~StageTimer() {
    if (a && b) {
      cudaEventRecord(b, st);
      c->pending.push_back({stage, a, b});
    } else {
      if (a) c->ev_free.push_back(a);
      if (b) c->ev_free.push_back(b);
    }
  }
};

void free_all(s2w_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
  for (cudaEvent_t e : c->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_out) cudaEventDestroy(e);
  c->ev_in.clear();
  c->ev_out.clear();
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  c->pending.clear();
  c->ev_free.clear();
  void* ps[] = {c->G, c->G_lo, c->G_scale, c->P, c->P_lo, c->tw_df, c->ws_shat_lo, c->ws_mhat_lo, c->ws_vhat_lo,
                c->ws_part_lo, c->tw, c->ws_slip, c->ws_shat, c->ws_mhat,
                c->ws_vhat, c->ws_part, c->ws_q, c->ws_seafloor, c->d_status, c->tc_bp1, c->ws_rhat, c->ws_gpart, c->ws_resid, c->ws_d, c->ws_loss,
                c->tc_mhat, c->tc_vhat, c->tc_part, c->tc_p2, c->tc_T, c->tc_bp1_lo, c->tc_vhat_lo, c->tc_p2_lo,
                c->tc_gT, c->tc_gT_lo, c->tc_pT, c->tc_pT_lo, c->tc_rb, c->tc_rb_lo, c->tc_ub, c->tc_ub_lo,
                c->tc_ghat, c->ws_lens, c->d_amax, c->tc_T_lo, c->tc_Ta, c->tc_Ta_lo, c->tc_colscale};
  for (void* p : ps)
    if (p) cudaFree(p);
}

// The retransform of one signal, vhat = FFT(ZeroPad(D_t(Truncate(IFFT(mhat))))),
// as a real 2 Nt x 2 Nt matrix T[n][k] over the degrees of freedom
// k = 0: Re bin 0, k = 1: Re bin Nt, k = 2l / 2l+1: Re / Im bin l (0 < l < Nt),
// the same ordering for the outputs n.  Column k is the map applied to basis
// spectrum k, evaluated in FP64 from the definitions (inverse DFT head,
// backward difference, or its transpose for the adjoint, zero-padded DFT);
// the caller rounds it to BF16 (hi, and lo = the rounded remainder for the
// split path).
std::vector<double> retransform_matrix(int Nt, int dt_mode, double dt, bool transpose = false) {
  const int L = 2 * Nt, K = 2 * Nt;
  std::vector<double> c(L), sn(L);
  for (int m = 0; m < L; ++m) {
    const double ang = 2.0 * 3.14159265358979323846 * m / L;
    c[m] = std::cos(ang);
    sn[m] = std::sin(ang);
  }
  std::vector<double> T(static_cast<size_t>(K) * K, 0.0), x(Nt), v(Nt);
  for (int k = 0; k < K; ++k) {
    for (int n = 0; n < Nt; ++n) {
      if (k == 0) x[n] = 1.0 / L;
      else if (k == 1) x[n] = (n % 2 == 0 ? 1.0 : -1.0) / L;
      else if (k % 2 == 0) x[n] = 2.0 / L * c[(static_cast<long long>(k / 2) * n) % L];
      else x[n] = -2.0 / L * sn[(static_cast<long long>(k / 2) * n) % L];
    }
    for (int n = 0; n < Nt; ++n) {
      if (dt_mode == S2W_DT_NONE)
        v[n] = x[n];
      else if (transpose)  // D_t^T: (w[n] - w[n+1]) / dt, w[Nt] = 0
        v[n] = (x[n] - (n + 1 < Nt ? x[n + 1] : 0.0)) / dt;
      else
        v[n] = (x[n] - (n > 0 ? x[n - 1] : 0.0)) / dt;
    }
    for (int l = 0; l <= Nt; ++l) {
      double re = 0.0, im = 0.0;
      for (int n = 0; n < Nt; ++n) {
        const long long m = (static_cast<long long>(n) * l) % L;
        re += v[n] * c[m];
        im -= v[n] * sn[m];
      }
      if (l == 0) T[0 * K + k] = re;
      else if (l == Nt) T[1 * K + k] = re;
      else {
        T[static_cast<size_t>(2 * l) * K + k] = re;
        T[static_cast<size_t>(2 * l + 1) * K + k] = im;
      }
    }
  }
  return T;
}

// Tensor-core pipeline for a batch of ruptures (slip and q device pointers),
// in sub-batches of at most tc_bsub ruptures:
//   rfft slip -> pack stage-1 B operand -> tcgen05 stage 1 -> mhat[l][b][Ng]
//   -> retransform (BF16 velocity spectra, the stage-2 A operand)
//   -> tcgen05 stage 2 over grid chunks -> partials -> reduce + IFFT -> q.
// One tcgen05 GEMM (epilogue 0: FP32 out[l][t][row]) over A [Nb][M][K]
// and the B operand rows [Nb][n_alloc][K] (BF16; lo parts when split).
// Stage-1 epilogue writing the BF16 (Re, Im) pairs the GEMM retransform
// reads to `dst`, [Nb][Bs][Ng_pad2], for Bs ruptures.
void set_pairs(s2w_ctx* ctx, TcArgs& a, int Bs, void* dst) {
  a.out = nullptr;
  a.out_bf = static_cast<__nv_bfloat162*>(dst);
  a.ld_t = ctx->Ng_pad2;
  a.ld_l = static_cast<long long>(Bs) * ctx->Ng_pad2;
}

// chunk_k > 0 (FP32 out): the K extent in launches of at most chunk_k
// elements each, in order, the first storing and the others adding their
// FP32 partial into `out` (each launch one FP32 accumulation of chunk_k
// terms at most).
int tc_gemm_epi0(s2w_ctx* ctx, const void* A, const void* A_lo, long long M, long long K, const void* Bop,
                 const void* B_lo, int n_alloc, int N, int T, float2* out, long long ld_l, long long ld_t,
                 cudaStream_t st, bool pairs = false, long long chunk_k = 0) {
  const int sp = A_lo != nullptr ? 1 : 0;
  CUtensorMap ta, tb, ta2, tb2;
  const int mt = static_cast<int>((M + 127) / 128);
  TcArgs a{};
  const int brows = tc_shape(a, N, mt, sp, 0, ctx->tc_pair);
  const int bk = tc_block_k(N, sp, a.cta2);
  CK(tc_encode_3d(&ta, A, K, M, ctx->Nb, K, 128, bk));
  CK(tc_encode_3d(&tb, Bop, K, n_alloc, ctx->Nb, K, brows, bk));
  if (sp) {
    CK(tc_encode_3d(&ta2, A_lo, K, M, ctx->Nb, K, 128, bk));
    CK(tc_encode_3d(&tb2, B_lo, K, n_alloc, ctx->Nb, K, brows, bk));
  }
  a.N = N;
  a.K = static_cast<int>(K);
  a.M_total = static_cast<int>(M);
  a.Nb = static_cast<int>(ctx->Nb);
  a.m_tiles = mt;
  a.n_kchunks = 1;
  a.kblocks_per_chunk = static_cast<int>((K + bk - 1) / bk);
  a.a_lo = sp;
  a.b_lo = sp;
  a.epi = 0;
  a.T = T;
  if (pairs) {
    set_pairs(ctx, a, T, out);
  } else {
    a.out = out;
    a.ld_l = ld_l;
    a.ld_t = ld_t;
  }
  a.status = ctx->d_status;
  const int nk = a.kblocks_per_chunk;
  const int per = chunk_k > 0 && !pairs ? static_cast<int>(std::max<long long>(1, chunk_k / bk)) : nk;
  for (int kb = 0; kb < nk; kb += per) {
    a.kb_off = kb;
    a.kblocks_per_chunk = std::min(per, nk - kb);
    a.acc_out = kb > 0 ? 1 : 0;
    CK(launch_tc_gemm(ta, tb, a, ctx->num_sms, st, sp ? &ta2 : nullptr, sp ? &tb2 : nullptr));
  }
  return S2W_OK;
}

// Adjoint of the waveform map on the tensor engine, per sub-batch (same
// steps as the streaming adjoint, each contraction one GEMM per bin):
//   rhat = rFFT(ZeroPad(r));  what_l = Phat_l^H rhat_l  (A = Phat_l^T, B = conj. embedding of rhat)
//   uhat = FFT(ZeroPad(D_t^T(Truncate(IFFT(what)))))      (FP32 FFT retransform, writes B directly)
//   ghat_l = Ghat_l^H uhat_l  (A = Ghat_l^T, K = grid);   g = Truncate(IFFT(ghat))
int adjoint_tensor(s2w_ctx* ctx, const float* r_d, int B, float* g_d, cudaStream_t st) {
  const long long Ns = ctx->Ns, Ng = ctx->Ng, No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb;
  const int sp = ctx->tc_split ? 1 : 0;
  const int dt_t = ctx->opts.dt_mode == S2W_DT_NONE ? S2W_DT_NONE : kDtTranspose;
  for (int b0 = 0; b0 < B; b0 += ctx->tc_bsub) {
    const int Bs = std::min(ctx->tc_bsub, B - b0);
    int N1 = static_cast<int>(round_up(2 * Bs, 16));
    if (N1 > 256) N1 = 512;
    {
      StageTimer t(ctx, 0, st);
      CK(launch_rfft_rows(r_d + static_cast<long long>(b0) * No * Nt, Bs * No, static_cast<int>(Nt),
                          static_cast<int>(Nt), ctx->tw, ctx->ws_rhat, Bs * No, No, No, st));
    }
    {
      StageTimer t(ctx, 6, st);
      CK(launch_pack_b(ctx->ws_rhat, static_cast<int>(Nb), Bs, No, static_cast<long long>(Bs) * No, No, 0, ctx->NoP,
                       ctx->tc_n1max, 1, ctx->tc_rb, ctx->tc_rb_lo, st));
    }
    float2* what = static_cast<float2*>(ctx->tc_mhat);
    // the GEMM retransform (D_t^T matrix) rounds what to BF16 anyway; the
    // split path keeps it in FP32 and splits it itself
    const bool gemm_rt = ctx->tc_Ta != nullptr;
    {
      StageTimer t(ctx, 3, st);
      int rc = tc_gemm_epi0(ctx, ctx->tc_pT, sp ? ctx->tc_pT_lo : nullptr, Ng, 2LL * ctx->NoP, ctx->tc_rb,
                            sp ? ctx->tc_rb_lo : nullptr, ctx->tc_n1max, N1, Bs, what,
                            static_cast<long long>(Bs) * Ng, Ng, st, gemm_rt && !sp);
      if (rc != S2W_OK) return rc;
    }
    if (gemm_rt) {  // uhat as the conjugate-embedding B operand: rows 2b, 2b+1 of [l][n1max][Ng_pad2]
      StageTimer t(ctx, 2, st);
      TcRtArgs r{};
      if (sp) {
        r.mhat32 = what;
        r.ld_l = static_cast<long long>(Bs) * Ng;
        r.ld_b = Ng;
      } else {
        r.mhat_bf = reinterpret_cast<const __nv_bfloat162*>(what);
        r.ld_l = static_cast<long long>(Bs) * ctx->Ng_pad2;
        r.ld_b = ctx->Ng_pad2;
      }
      r.Ng = static_cast<int>(Ng);
      r.Bs = Bs;
      r.Nt = static_cast<int>(Nt);
      r.vhat = static_cast<__nv_bfloat162*>(ctx->tc_ub);
      r.vhat_lo = static_cast<__nv_bfloat162*>(ctx->tc_ub_lo);
      r.vld_l = static_cast<long long>(ctx->tc_n1max) * ctx->Ng_pad2;
      r.vld_b = 2 * ctx->Ng_pad2;
      r.conj_row = ctx->Ng_pad2;
      r.status = ctx->d_status;
      CK(launch_tc_retransform(ctx->tc_tmTa, sp ? &ctx->tc_tmTa2 : nullptr, r, ctx->num_sms, st,
                               sp || !ctx->tc_rtpair ? nullptr : &ctx->tc_tmTap));
    } else {
      StageTimer t(ctx, 2, st);
      CK(launch_retransform(what, Ng, static_cast<long long>(Bs) * Ng, static_cast<int>(Nt), ctx->tw,
                            static_cast<float>(1.0 / ctx->opts.dt), dt_t, nullptr, ctx->Ng_pad2, nullptr, st, Bs, Ng, 0,
                            static_cast<__nv_bfloat162*>(ctx->tc_ub), static_cast<__nv_bfloat162*>(ctx->tc_ub_lo),
                            ctx->tc_n1max));
    }
    {
      StageTimer t(ctx, 1, st);
      // K = the grid: the split precision keeps each FP32 accumulation
      // within kSplitAdjChunkK terms
      int rc = tc_gemm_epi0(ctx, ctx->tc_gT, sp ? ctx->tc_gT_lo : nullptr, Ns, 2 * ctx->Ng_pad2, ctx->tc_ub,
                            sp ? ctx->tc_ub_lo : nullptr, ctx->tc_n1max, N1, Bs, ctx->tc_ghat,
                            static_cast<long long>(Bs) * Ns, Ns, st, false, sp ? kSplitAdjChunkK : 0);
      if (rc != S2W_OK) return rc;
    }
    {
      StageTimer t(ctx, 4, st);
      CK(launch_reduce_irfft(ctx->tc_ghat, Bs, static_cast<int>(Ns), 1, static_cast<int>(Nt), Ns,
                             static_cast<long long>(Bs) * Ns, 0, ctx->tw, g_d + static_cast<long long>(b0) * Ns * Nt,
                             st));
    }
  }
  return S2W_OK;
}

int waveforms_tensor(s2w_ctx* ctx, const float* slip_d, int B, float* q_d, cudaStream_t st) {
  const long long Ns = ctx->Ns, Ng = ctx->Ng, No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb, Ns_pad = ctx->Ns_pad;
  const int K1 = static_cast<int>(2 * Ns_pad);
  const long long K2 = 2 * ctx->Ng_pad2;
  for (int b0 = 0; b0 < B; b0 += ctx->tc_bsub) {
    const int Bs = std::min(ctx->tc_bsub, B - b0);
    const int m1 = static_cast<int>((Ng + 127) / 128);
    const int sp = ctx->tc_split ? 1 : 0;
    const bool f8 = ctx->opts.prec_g == S2W_PREC_FP8_E4M3;
    // FP8 x FP8 stage 1 (two-SM tiles: N % 32, at least two M tiles)
    const bool f8f8 = f8 && ctx->tc_f8act && m1 >= 2;
    int N1 = static_cast<int>(round_up(2 * Bs, f8f8 ? 32 : 16));
    if (N1 > 256) N1 = 512;
    {
      StageTimer t(ctx, 0, st);
      CK(launch_rfft_rows(slip_d + static_cast<long long>(b0) * Ns * Nt, Bs * Ns, static_cast<int>(Nt),
                          static_cast<int>(Nt), ctx->tw, ctx->ws_shat, Bs * Ns_pad, Ns, Ns_pad, st,
                          ctx->cur_lens ? ctx->cur_lens + b0 : nullptr));
    }
    {
      StageTimer t(ctx, 6, st, f8 && !f8f8 ? 2 : 1);
      if (f8f8)  // e4m3 operand (+ lo parts), one power-of-two scale per (bin, rupture)
        CK(launch_pack_b_f8(ctx->ws_shat, static_cast<int>(Nb), Bs, Ns_pad, static_cast<long long>(Bs) * Ns_pad,
                            Ns_pad, Ns_pad, ctx->tc_n1max, N1, ctx->tc_colscale, ctx->tc_n1max / 2, ctx->tc_bp1,
                            ctx->tc_f8lo ? ctx->tc_bp1_lo : nullptr, st));
      else if (f8)  // FP16 operand for the FP16 MMAs of the FP8 path, scaled by a power of two from its amax
        CK(launch_pack_b_f16(ctx->ws_shat, static_cast<int>(Nb), Bs, Ns_pad, static_cast<long long>(Bs) * Ns_pad,
                             Ns_pad, Ns_pad, ctx->tc_n1max, ctx->d_amax, ctx->tc_bp1, st));
      else
        CK(launch_pack_b(ctx->ws_shat, static_cast<int>(Nb), Bs, Ns_pad, static_cast<long long>(Bs) * Ns_pad, Ns_pad,
                         0, Ns_pad, ctx->tc_n1max, 0, ctx->tc_bp1, ctx->tc_bp1_lo, st));
    }
    if (f8f8) {
      StageTimer t(ctx, 1, st);
      CUtensorMap ta, tb, tb2;
      // byte maps: K blocks of 128 e4m3 elements with 128-byte swizzle, or
      // of 64 with 64-byte swizzle when B comes as hi + lo parts of up to
      // 256 columns; hi + lo at N = 512: each unit takes one 256-column
      // half (n_split), and two accumulators alternate in tensor memory
      const bool lo = ctx->tc_f8lo;
      const bool nsp = lo && N1 == 512;
      const int bkb = lo && !nsp ? 64 : 128;
      const int swz = lo && !nsp ? 2 : 1;
      const int brows = (N1 > 256 ? 256 : N1) / 2;
      CK(tc_encode_3d_u8(&ta, ctx->G, K1, Ng, Nb, 128, bkb, swz));
      CK(tc_encode_3d_u8(&tb, ctx->tc_bp1, K1, ctx->tc_n1max, Nb, brows, bkb, swz));
      if (lo) CK(tc_encode_3d_u8(&tb2, ctx->tc_bp1_lo, K1, ctx->tc_n1max, Nb, brows, bkb, swz));
      TcArgs a{};
      a.N = N1;
      a.K = K1;
      a.M_total = static_cast<int>(Ng);
      a.Nb = static_cast<int>(Nb);
      a.m_tiles = m1;
      a.n_kchunks = 1;
      a.kblocks_per_chunk = (K1 + bkb - 1) / bkb;
      a.cta2 = 1;
      a.stages = tc_stages_pair(nsp ? N1 / 2 : N1, 0, lo ? (nsp ? 4 : 3) : 2);
      a.n_split = nsp ? 2 : 1;
      a.tmem_cols = N1 <= 32 ? 32 : (N1 <= 64 ? 64 : (N1 <= 128 ? 128 : (N1 <= 256 ? 256 : 512)));
      a.a_fp8 = 1;
      a.row_scale = ctx->G_scale;
      a.nblk = ctx->nblk;
      a.epi = 0;
      a.T = Bs;
      set_pairs(ctx, a, Bs, ctx->tc_mhat);
      a.status = ctx->d_status;
      CK(launch_tc_gemm(ta, tb, a, ctx->num_sms, st, nullptr, lo ? &tb2 : nullptr, ctx->tc_colscale,
                        ctx->tc_n1max / 2));
    } else {
      StageTimer t(ctx, 1, st);
      CUtensorMap ta, tb, ta2, tb2;
      TcArgs a{};
      const int brows = tc_shape(a, N1, m1, sp, f8 ? 1 : 0, ctx->tc_pair);
      const int bk = tc_block_k(N1, sp, a.cta2);
      if (f8)  // one byte per K element: row pitch 2 Ns_pad bytes
        CK(tc_encode_3d_u8(&ta, ctx->G, K1, Ng, Nb, 128, bk));
      else
        CK(tc_encode_3d(&ta, ctx->G, K1, Ng, Nb, K1, 128, bk));
      CK(tc_encode_3d(&tb, ctx->tc_bp1, K1, ctx->tc_n1max, Nb, K1, brows, bk));
      if (sp) {
        CK(tc_encode_3d(&ta2, ctx->G_lo, K1, Ng, Nb, K1, 128, bk));
        CK(tc_encode_3d(&tb2, ctx->tc_bp1_lo, K1, ctx->tc_n1max, Nb, K1, brows, bk));
      }
      a.N = N1;
      a.K = K1;
      a.M_total = static_cast<int>(Ng);
      a.Nb = static_cast<int>(Nb);
      a.m_tiles = static_cast<int>((Ng + 127) / 128);
      a.n_kchunks = 1;
      a.kblocks_per_chunk = (K1 + bk - 1) / bk;
      a.a_lo = sp;
      a.b_lo = sp;
      a.a_fp8 = f8 ? 1 : 0;
      if (f8) {  // FP8 rows carry one scale per (bin, 256 grid rows); B its power-of-two scale
        a.row_scale = ctx->G_scale;
        a.nblk = ctx->nblk;
        a.b_amax = ctx->d_amax;
      }
      a.epi = 0;
      a.T = Bs;
      // the GEMM retransform rounds the seafloor spectra to BF16 anyway (BF16
      // pairs, its TMA operand); the split path keeps them in FP32 and
      // splits them into hi + lo itself
      if (sp) {
        a.out = static_cast<float2*>(ctx->tc_mhat);
        a.ld_l = static_cast<long long>(Bs) * Ng;
        a.ld_t = Ng;
      } else {
        set_pairs(ctx, a, Bs, ctx->tc_mhat);
      }
      a.status = ctx->d_status;
      CK(launch_tc_gemm(ta, tb, a, ctx->num_sms, st, sp ? &ta2 : nullptr, sp ? &tb2 : nullptr));
    }
    {
      StageTimer t(ctx, 2, st);
      TcRtArgs r{};
      if (sp) {
        r.mhat32 = static_cast<const float2*>(ctx->tc_mhat);
        r.ld_l = static_cast<long long>(Bs) * Ng;
        r.ld_b = Ng;
      } else {
        r.mhat_bf = reinterpret_cast<const __nv_bfloat162*>(ctx->tc_mhat);
        r.ld_l = static_cast<long long>(Bs) * ctx->Ng_pad2;
        r.ld_b = ctx->Ng_pad2;
      }
      r.vhat_lo = static_cast<__nv_bfloat162*>(ctx->tc_vhat_lo);
      r.Ng = static_cast<int>(Ng);
      r.Bs = Bs;
      r.Nt = static_cast<int>(Nt);
      r.vhat = static_cast<__nv_bfloat162*>(ctx->tc_vhat);
      r.vld_l = static_cast<long long>(ctx->tc_bsub) * ctx->Ng_pad2;
      r.vld_b = ctx->Ng_pad2;
      r.status = ctx->d_status;
      CK(launch_tc_retransform(ctx->tc_tmT, sp ? &ctx->tc_tmT2 : nullptr, r, ctx->num_sms, st,
                               sp || !ctx->tc_rtpair ? nullptr : &ctx->tc_tmTp));
    }
    {
      StageTimer t(ctx, 3, st);
      CUtensorMap ta, tb, ta2, tb2;
      const int m2 = (Bs + 127) / 128;
      TcArgs a{};
      // the half-stored operand runs on one CTA per tile (or M-tile pair)
      int brows = tc_shape(a, ctx->tc_n2, m2, sp, 0, ctx->tc_p2h ? 0 : ctx->tc_pair);
      // the chunk length tc_kbpc counts K blocks of the single-CTA size
      if (tc_block_k(ctx->tc_n2, sp, a.cta2) != tc_block_k(ctx->tc_n2, sp)) brows = tc_shape(a, ctx->tc_n2, m2, sp, 0, 0);
      const int bk = tc_block_k(ctx->tc_n2, sp, a.cta2);
      const int p2rows = ctx->tc_p2h ? ctx->tc_n2 / 2 : ctx->tc_n2;
      a.b_half = ctx->tc_p2h ? 1 : 0;
      CK(tc_encode_3d(&ta, ctx->tc_vhat, K2, ctx->tc_bsub, Nb, K2, 128, bk));
      CK(tc_encode_3d(&tb, ctx->tc_p2, K2, p2rows, Nb, K2, ctx->tc_p2h ? p2rows : brows, bk));
      if (sp) {
        CK(tc_encode_3d(&ta2, ctx->tc_vhat_lo, K2, ctx->tc_bsub, Nb, K2, 128, bk));
        CK(tc_encode_3d(&tb2, ctx->tc_p2_lo, K2, ctx->tc_n2, Nb, K2, brows, bk));
      }
      a.N = ctx->tc_n2;
      a.K = static_cast<int>(K2);
      a.M_total = Bs;
      a.Nb = static_cast<int>(Nb);
      a.m_tiles = (Bs + 127) / 128;
      a.n_kchunks = ctx->tc_nkc;
      a.kblocks_per_chunk = ctx->tc_kbpc;
      a.a_lo = sp;
      a.b_lo = sp;
      a.epi = 1;
      a.T = static_cast<int>(No);
      a.out = ctx->tc_part;
      a.status = ctx->d_status;
      CK(launch_tc_gemm(ta, tb, a, ctx->num_sms, st, sp ? &ta2 : nullptr, sp ? &tb2 : nullptr));
    }
    {
      StageTimer t(ctx, 4, st);
      // many chunks (the split precision): add them up first along the
      // contiguous (rupture, observation) rows, in the same order
      int nseg = ctx->tc_nkc;
      if (nseg > 8) {
        CK(launch_sum_chunks(ctx->tc_part, static_cast<int>(Nb), nseg, static_cast<long long>(Bs) * No, st));
        nseg = 1;
      }
      CK(launch_reduce_irfft(ctx->tc_part, Bs, static_cast<int>(No), nseg, static_cast<int>(Nt), No,
                             static_cast<long long>(ctx->tc_nkc) * Bs * No, static_cast<long long>(Bs) * No, ctx->tw,
                             q_d + static_cast<long long>(b0) * No * Nt, st));
    }
  }
  return S2W_OK;
}

}  // namespace

extern "C" {

int s2w_retransform_matrix(int Nt, int dt_mode, double dt, int transpose, double* T) {
  if (T == nullptr) return fail(nullptr, S2W_ERR_ARG, "retransform_matrix: T is NULL");
  if (Nt != 32 && Nt != 64 && Nt != 128 && Nt != 256)
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "retransform_matrix: Nt=%d: supported 32, 64, 128, 256", Nt);
  if (dt_mode != S2W_DT_BACKWARD && dt_mode != S2W_DT_NONE)
    return fail(nullptr, S2W_ERR_ARG, "retransform_matrix: dt_mode=%d", dt_mode);
  if (!(dt > 0.0)) return fail(nullptr, S2W_ERR_ARG, "retransform_matrix: dt must be > 0");
  if (transpose != 0 && transpose != 1) return fail(nullptr, S2W_ERR_ARG, "retransform_matrix: transpose=%d", transpose);
  const std::vector<double> M = retransform_matrix(Nt, dt_mode, dt, transpose != 0);
  std::copy(M.begin(), M.end(), T);
  return S2W_OK;
}

void s2w_default_opts(s2w_opts* o) {
  if (!o) return;
  o->prec_g = S2W_PREC_FP32;
  o->prec_p = S2W_PREC_FP32;
  o->dt_mode = S2W_DT_BACKWARD;
  o->dt = 1.0;
  o->max_batch = 1;
  o->device = 0;
  o->engine = S2W_ENGINE_AUTO;
  o->tc_adjoint = 0;
  o->single_pass = 0;
  o->tc_pair = S2W_PAIR_AUTO;
  o->tc_fp8_act = 2;
  o->tc_bsub = 0;
  o->tc_s2_chunks = 0;
  o->tune_cache = nullptr;
  o->fault = S2W_FAULT_NONE;
  o->fault_wait_us = 5000;
}

const char* s2w_status_string(int s) {
  switch (s) {
    case S2W_OK: return "S2W_OK";
    case S2W_ERR_ARG: return "S2W_ERR_ARG";
    case S2W_ERR_OOM: return "S2W_ERR_OOM";
    case S2W_ERR_STATE: return "S2W_ERR_STATE";
    case S2W_ERR_CUDA: return "S2W_ERR_CUDA";
    case S2W_ERR_TIMEOUT: return "S2W_ERR_TIMEOUT";
    case S2W_ERR_UNSUPPORTED: return "S2W_ERR_UNSUPPORTED";
    default: return "S2W_ERR_UNKNOWN";
  }
}

const char* s2w_last_error(const s2w_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

int s2w_create(int Ns, int Ng, int No, int Nt, const s2w_opts* opts, s2w_ctx** out) {
  s2w_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, S2W_ERR_ARG, "out is NULL");
  *out = nullptr;
  s2w_opts o;
  s2w_default_opts(&o);
  if (opts) o = *opts;
  if (Ns < 1 || Ng < 1 || No < 1) return fail(nullptr, S2W_ERR_ARG, "Ns, Ng, No must be >= 1");
  if (!supported_nt(Nt)) return fail(nullptr, S2W_ERR_UNSUPPORTED, "Nt=%d: supported 32, 64, 128, 256, 512", Nt);
  if (Ns > 1024) return fail(nullptr, S2W_ERR_UNSUPPORTED, "Ns=%d > 1024", Ns);
  if (o.prec_g < S2W_PREC_FP32 || o.prec_g > S2W_PREC_FP32_HILO)
    return fail(nullptr, S2W_ERR_ARG, "prec_g=%d", o.prec_g);
  if (o.prec_p != S2W_PREC_FP32 && o.prec_p != S2W_PREC_BF16 && o.prec_p != S2W_PREC_FP32_HILO)
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "prec_p=%d: FP32, BF16 or FP32_HILO", o.prec_p);
  if ((o.prec_g == S2W_PREC_FP32_HILO) != (o.prec_p == S2W_PREC_FP32_HILO))
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "prec_g=%d, prec_p=%d: FP32_HILO is for both operators or neither",
                o.prec_g, o.prec_p);
  if (o.prec_g == S2W_PREC_FP32_HILO && (o.engine == S2W_ENGINE_TENSOR || o.single_pass || o.tc_adjoint))
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "FP32_HILO: stream engine only, no single_pass or tc_adjoint");
  if (o.dt_mode != S2W_DT_BACKWARD && o.dt_mode != S2W_DT_NONE)
    return fail(nullptr, S2W_ERR_ARG, "dt_mode=%d", o.dt_mode);
  if (!(o.dt > 0.0)) return fail(nullptr, S2W_ERR_ARG, "dt must be > 0");
  if (o.max_batch < 1) return fail(nullptr, S2W_ERR_ARG, "max_batch must be >= 1");
  if (o.engine < S2W_ENGINE_AUTO || o.engine > S2W_ENGINE_TENSOR) return fail(nullptr, S2W_ERR_ARG, "engine=%d", o.engine);
  if (o.tc_bsub != 0 && o.tc_bsub != 128 && o.tc_bsub != 256)
    return fail(nullptr, S2W_ERR_ARG, "tc_bsub=%d: 0, 128 or 256", o.tc_bsub);
  if (o.tc_bsub == 256 && o.prec_g == S2W_PREC_BF16_HILO)
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "tc_bsub=256: split (BF16_HILO) passes take at most 128 ruptures");
  if (o.tc_s2_chunks < 0 || o.tc_s2_chunks > kMaxS2Chunks)
    return fail(nullptr, S2W_ERR_ARG, "tc_s2_chunks=%d: 0..%d", o.tc_s2_chunks, kMaxS2Chunks);
  if (o.fault < S2W_FAULT_NONE || o.fault > S2W_FAULT_LAUNCH) return fail(nullptr, S2W_ERR_ARG, "fault=%d", o.fault);
  if (o.fault == S2W_FAULT_NONE) {  // test hook from the environment
    const char* f = std::getenv("S2W_FAULT");
    if (f && std::strcmp(f, "wait") == 0) o.fault = S2W_FAULT_WAIT;
    else if (f && std::strcmp(f, "oom_load") == 0) o.fault = S2W_FAULT_OOM_LOAD;
    else if (f && std::strcmp(f, "launch") == 0) o.fault = S2W_FAULT_LAUNCH;
    else if (f && *f) return fail(nullptr, S2W_ERR_ARG, "S2W_FAULT=%s: wait, oom_load or launch", f);
  }
  if (o.fault == S2W_FAULT_WAIT && (o.fault_wait_us < 1 || o.fault_wait_us > 2000000))
    return fail(nullptr, S2W_ERR_ARG, "fault_wait_us=%d: 1..2000000", o.fault_wait_us);
  if (o.engine == S2W_ENGINE_TENSOR && o.prec_g == S2W_PREC_FP32)
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "the tensor engine needs prec_g = BF16, BF16_HILO or FP8_E4M3");
  if (o.tc_adjoint != 0 && o.tc_adjoint != 1) return fail(nullptr, S2W_ERR_ARG, "tc_adjoint=%d: 0 or 1", o.tc_adjoint);
  if (o.single_pass != 0 && o.single_pass != 1)
    return fail(nullptr, S2W_ERR_ARG, "single_pass=%d: 0 or 1", o.single_pass);
  if (o.tc_pair != S2W_PAIR_AUTO && o.tc_pair != S2W_PAIR_ON && o.tc_pair != S2W_PAIR_OFF)
    return fail(nullptr, S2W_ERR_ARG, "tc_pair=%d: S2W_PAIR_AUTO, _ON or _OFF", o.tc_pair);
  if (o.tc_fp8_act < 0 || o.tc_fp8_act > 2)
    return fail(nullptr, S2W_ERR_ARG, "tc_fp8_act=%d: 0, 1 or 2", o.tc_fp8_act);
  if (o.tc_fp8_act && o.prec_g != S2W_PREC_FP8_E4M3) {
    if (!opts || o.tc_fp8_act == 2) o.tc_fp8_act = 0;  // the default applies to FP8 operators only
    else return fail(nullptr, S2W_ERR_ARG, "tc_fp8_act needs prec_g = S2W_PREC_FP8_E4M3");
  }
  if (o.single_pass && (Nt > 256 || o.engine == S2W_ENGINE_TENSOR || o.tc_adjoint))
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "single_pass: stream engine only, Nt <= 256, no tc_adjoint");
  if (o.engine == S2W_ENGINE_TENSOR && 2 * No > 256)
    return fail(nullptr, S2W_ERR_UNSUPPORTED, "the tensor engine needs No <= 128");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, S2W_ERR_CUDA, "no CUDA device %d", o.device);
  }
  DeviceGuard guard(o.device);
  ctx = new s2w_ctx();
  ctx->Ns = Ns;
  ctx->Ng = Ng;
  ctx->No = No;
  ctx->Nt = Nt;
  // single pass: L = 4 Nt >= 3 Nt - 1 (no wrap without the retransform)
  ctx->single_pass = o.single_pass != 0;
  ctx->Nb = ctx->single_pass ? 2 * Nt + 1 : Nt + 1;
  ctx->L = ctx->single_pass ? 4 * Nt : 2 * Nt;
  ctx->Ns_pad = static_cast<int>(round_up(Ns, 8));
  ctx->nseg = static_cast<int>((Ng + 1023) / 1024);
  ctx->RL = static_cast<int>(round_up((Ng + ctx->nseg - 1) / ctx->nseg, 8));
  ctx->opts = o;
  ctx->opts.tune_cache = nullptr;  // the caller's string is not kept
  if (o.tune_cache) ctx->tune_cache = o.tune_cache;
  ctx->fault = o.fault;
  if (o.fault == S2W_FAULT_WAIT) ctx->wait_ns = 1000ull * static_cast<unsigned long long>(o.fault_wait_us);
  ctx->device = o.device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, o.device);
  ctx->g_loaded.assign(Ng, 0);
  ctx->p_loaded.assign(Ng, 0);

  const long long Nb = ctx->Nb, B = o.max_batch;
  const size_t gcb = elem_complex_bytes(o.prec_g);
  ctx->nblk = static_cast<int>((Ng + 255) / 256);
  ctx->g_bytes = static_cast<size_t>(Nb) * Ng * ctx->Ns_pad * gcb;
  ctx->df = o.prec_g == S2W_PREC_FP32_HILO;
  if (o.prec_g == S2W_PREC_BF16_HILO || ctx->df) ctx->g_bytes *= 2;
  if (o.prec_g == S2W_PREC_FP8_E4M3) ctx->g_bytes += static_cast<size_t>(Nb) * ctx->nblk * sizeof(float);
  const size_t psz = static_cast<size_t>(Nb) * ctx->nseg * No * ctx->RL * elem_complex_bytes(o.prec_p);
  ctx->p_bytes = psz * (ctx->df ? 2 : 1);

  auto bad = [&](cudaError_t e, const char* what) {
    fail(nullptr, e == cudaErrorMemoryAllocation ? S2W_ERR_OOM : S2W_ERR_CUDA, "%s: %s", what,
         cudaGetErrorString(e));
    free_all(ctx);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? S2W_ERR_OOM : S2W_ERR_CUDA;
  };
  cudaError_t e;
  const size_t gsz = static_cast<size_t>(Nb) * Ng * ctx->Ns_pad * gcb;
  if ((e = dalloc(&ctx->G, gsz)) != cudaSuccess) return bad(e, "Ghat");
  if ((o.prec_g == S2W_PREC_BF16_HILO || ctx->df) && (e = dalloc(&ctx->G_lo, gsz)) != cudaSuccess)
    return bad(e, "Ghat lo");
  if (o.prec_g == S2W_PREC_FP8_E4M3 &&
      (e = dalloc(&ctx->G_scale, static_cast<size_t>(Nb) * ctx->nblk * sizeof(float))) != cudaSuccess)
    return bad(e, "Ghat scales");
  if ((e = dalloc(&ctx->P, psz)) != cudaSuccess) return bad(e, "Phat");
  if (ctx->df) {
    if ((e = dalloc(&ctx->P_lo, psz)) != cudaSuccess) return bad(e, "Phat lo");
    if ((e = dalloc(&ctx->tw_df, sizeof(float4) * ctx->L)) != cudaSuccess) return bad(e, "pair twiddles");
    const long long Bsh = std::min<long long>(B, kStreamGroup);
    if ((e = dalloc(&ctx->ws_shat_lo, sizeof(float2) * Nb * Bsh * ctx->Ns_pad)) != cudaSuccess)
      return bad(e, "slip spectra lo");
    if ((e = dalloc(&ctx->ws_mhat_lo, sizeof(float2) * Nb * Ng)) != cudaSuccess) return bad(e, "seafloor spectra lo");
    if ((e = dalloc(&ctx->ws_vhat_lo, sizeof(float2) * Nb * ctx->nseg * ctx->RL)) != cudaSuccess)
      return bad(e, "velocity spectra lo");
    if ((e = dalloc(&ctx->ws_part_lo, sizeof(float2) * Bsh * Nb * ctx->nseg * No)) != cudaSuccess)
      return bad(e, "stage-2 partials lo");
  }
  if ((e = dalloc(&ctx->tw, sizeof(float2) * ctx->L)) != cudaSuccess) return bad(e, "twiddles");
  if ((e = dalloc(&ctx->ws_slip, sizeof(float) * B * Ns * Nt)) != cudaSuccess) return bad(e, "slip workspace");
  const long long Bsh = std::min<long long>(B, 256);  // slip spectra serve one group / sub-batch at a time
  if ((e = dalloc(&ctx->ws_shat, sizeof(float2) * Nb * Bsh * ctx->Ns_pad)) != cudaSuccess)
    return bad(e, "slip spectra");
  if ((e = dalloc(&ctx->ws_mhat, sizeof(float2) * Nb * Ng)) != cudaSuccess) return bad(e, "seafloor spectra");
  if ((e = dalloc(&ctx->ws_vhat, sizeof(float2) * Nb * ctx->nseg * ctx->RL)) != cudaSuccess)
    return bad(e, "velocity spectra");
  if ((e = dalloc(&ctx->ws_part, sizeof(float2) * std::min<long long>(B, kStreamGroup) * Nb * ctx->nseg * No)) !=
      cudaSuccess)
    return bad(e, "stage-2 partials");
  if ((e = dalloc(&ctx->ws_q, sizeof(float) * B * No * Nt)) != cudaSuccess) return bad(e, "waveform workspace");
  if ((e = dalloc(&ctx->ws_seafloor, sizeof(float) * static_cast<size_t>(Ng) * Nt)) != cudaSuccess)
    return bad(e, "seafloor workspace");
  if ((e = dalloc(&ctx->d_status, sizeof(int))) != cudaSuccess) return bad(e, "status word");
  ctx->adj_nchunk = static_cast<int>((Ng + ctx->adj_rc - 1) / ctx->adj_rc);
  if ((e = dalloc(&ctx->ws_rhat, sizeof(float2) * Nb * B * No)) != cudaSuccess) return bad(e, "residual spectra");
  if ((e = dalloc(&ctx->ws_resid, sizeof(float) * B * No * Nt)) != cudaSuccess) return bad(e, "residuals");
  if ((e = dalloc(&ctx->ws_d, sizeof(float) * B * No * Nt)) != cudaSuccess) return bad(e, "targets");
  if ((e = dalloc(&ctx->ws_loss, sizeof(float) * B)) != cudaSuccess) return bad(e, "losses");
  if ((e = dalloc(&ctx->ws_lens, sizeof(int) * B)) != cudaSuccess) return bad(e, "active lengths");
  if ((e = dalloc(&ctx->d_amax, sizeof(unsigned))) != cudaSuccess) return bad(e, "operand range word");
  if ((e = dalloc(&ctx->ws_gpart, sizeof(float2) * Nb * ctx->adj_nchunk * ctx->Ns_pad)) != cudaSuccess)
    return bad(e, "adjoint partials");
  // AUTO keeps the tensor engine ready at any max_batch: single ruptures go
  // to it only if s2w_autotune measured it faster (tc_min_batch = 1)
  ctx->tc_on = !ctx->single_pass && o.prec_g != S2W_PREC_FP32 && !ctx->df && 2 * No <= 256 &&
               (o.engine == S2W_ENGINE_TENSOR || o.engine == S2W_ENGINE_AUTO);
  ctx->tc_split = ctx->tc_on && o.prec_g == S2W_PREC_BF16_HILO;
  if (ctx->tc_on) {
    // split operands double the B tiles: sub-batches of up to 128 ruptures
    const int bsub_want = o.tc_bsub > 0 ? o.tc_bsub : (ctx->tc_split ? 128 : 256);
    ctx->tc_bsub = static_cast<int>(std::min<long long>(B, bsub_want));
    ctx->tc_bsub_max = ctx->tc_bsub;
    ctx->tc_pair = o.tc_pair == S2W_PAIR_ON ? 1 : (o.tc_pair == S2W_PAIR_OFF ? 0 : kDefaultPair);
    // the two-SM retransform measured slower (9.0 against 8.4 ms per 256-rupture
    // batch): only when asked for
    ctx->tc_rtpair = o.tc_pair == S2W_PAIR_ON;
    ctx->tc_f8act = o.tc_fp8_act != 0;
    ctx->tc_f8lo = o.tc_fp8_act == 2;
    // FP8 B rows come in multiples of 32 (N % 32 for the two-SM tiles)
    ctx->tc_n1max = static_cast<int>(round_up(2 * ctx->tc_bsub, ctx->tc_f8act ? 32 : 16));
    if (ctx->tc_n1max > 256) ctx->tc_n1max = 512;
    // BF16 stage 2 stores each adjoint spectrum once (b_half: the converter
    // warps build the embedding's second row per stage); the split keeps
    // both rows of hi and lo
    ctx->tc_p2h = !ctx->tc_split;
    ctx->tc_n2 = static_cast<int>(ctx->tc_p2h ? 2 * round_up(No, 16) : round_up(2 * No, 16));
    ctx->Ng_pad2 = round_up(Ng, 8);
    ctx->s2_max_chunks = kMaxS2Chunks;
    if (ctx->tc_split) {
      const int bk2 = tc_block_k(ctx->tc_n2, 1);
      const long long k2 = (2 * ctx->Ng_pad2 + bk2 - 1) / bk2 * bk2;
      ctx->s2_min_chunks = static_cast<int>((k2 + kSplitChunkK - 1) / kSplitChunkK);
      ctx->s2_max_chunks = std::max(kMaxS2Chunks, ctx->s2_min_chunks);
    }
    set_s2_chunks(ctx, o.tc_s2_chunks);
    const long long bs = ctx->tc_bsub;
    const bool sp = ctx->tc_split;
    if ((e = dalloc(&ctx->tc_bp1, 2ull * Nb * ctx->tc_n1max * 2 * ctx->Ns_pad)) != cudaSuccess)
      return bad(e, "tensor stage-1 operand");
    if (ctx->tc_f8act &&
        (e = dalloc(&ctx->tc_colscale, sizeof(float) * Nb * (ctx->tc_n1max / 2))) != cudaSuccess)
      return bad(e, "FP8 activation scales");
    if (ctx->tc_f8lo && (e = dalloc(&ctx->tc_bp1_lo, 1ull * Nb * ctx->tc_n1max * 2 * ctx->Ns_pad)) != cudaSuccess)
      return bad(e, "FP8 activation low-order parts");
    ctx->tc_adj = o.tc_adjoint != 0;
    // FP32 seafloor spectra for the split path, and for the adjoint's what
    const bool mhat32 = sp || ctx->tc_adj;
    const size_t mh_pairs = sizeof(__nv_bfloat162) * Nb * bs * ctx->Ng_pad2;  // the BF16 retransform's TMA operand
    if ((e = dalloc(&ctx->tc_mhat, std::max<size_t>((mhat32 ? sizeof(float2) * Nb * bs * Ng : 0), mh_pairs))) !=
        cudaSuccess)
      return bad(e, "tensor seafloor spectra");
    if (ctx->tc_adj) {
      ctx->NoP = static_cast<int>(round_up(No, 32));
      const size_t gT = 4ull * Nb * Ns * round_up(Ng, 8), pT = 4ull * Nb * Ng * ctx->NoP;
      const size_t rb = 2ull * Nb * ctx->tc_n1max * 2 * ctx->NoP;
      const size_t ub = 2ull * Nb * ctx->tc_n1max * 2 * round_up(Ng, 8);
      if ((e = dalloc(&ctx->tc_gT, gT)) != cudaSuccess) return bad(e, "transposed Ghat");
      if ((e = dalloc(&ctx->tc_pT, pT)) != cudaSuccess) return bad(e, "transposed Phat");
      if ((e = dalloc(&ctx->tc_rb, rb)) != cudaSuccess) return bad(e, "adjoint residual operand");
      if ((e = dalloc(&ctx->tc_ub, ub)) != cudaSuccess) return bad(e, "adjoint stage-1 operand");
      if (sp) {
        if ((e = dalloc(&ctx->tc_gT_lo, gT)) != cudaSuccess) return bad(e, "transposed Ghat (lo)");
        if ((e = dalloc(&ctx->tc_pT_lo, pT)) != cudaSuccess) return bad(e, "transposed Phat (lo)");
        if ((e = dalloc(&ctx->tc_rb_lo, rb)) != cudaSuccess) return bad(e, "adjoint residual operand (lo)");
        if ((e = dalloc(&ctx->tc_ub_lo, ub)) != cudaSuccess) return bad(e, "adjoint stage-1 operand (lo)");
      }
      if ((e = dalloc(&ctx->tc_ghat, sizeof(float2) * Nb * bs * Ns)) != cudaSuccess)
        return bad(e, "adjoint slip spectra");
      ctx->g_bytes += gT * (sp ? 2 : 1);
      ctx->p_bytes += pT * (sp ? 2 : 1);
    }
    if ((e = dalloc(&ctx->tc_vhat, 4ull * Nb * bs * ctx->Ng_pad2)) != cudaSuccess)
      return bad(e, "tensor velocity spectra");
    if ((e = dalloc(&ctx->tc_part, sizeof(float2) * Nb * ctx->s2_max_chunks * bs * No)) != cudaSuccess)
      return bad(e, "tensor stage-2 partials");
    if ((e = dalloc(&ctx->tc_p2, 4ull * Nb * (ctx->tc_p2h ? ctx->tc_n2 / 2 : ctx->tc_n2) * ctx->Ng_pad2)) !=
        cudaSuccess)
      return bad(e, "tensor stage-2 operand");
    if (sp) {
      if ((e = dalloc(&ctx->tc_bp1_lo, 2ull * Nb * ctx->tc_n1max * 2 * ctx->Ns_pad)) != cudaSuccess)
        return bad(e, "tensor stage-1 operand (lo)");
      if ((e = dalloc(&ctx->tc_vhat_lo, 4ull * Nb * bs * ctx->Ng_pad2)) != cudaSuccess)
        return bad(e, "tensor velocity spectra (lo)");
      if ((e = dalloc(&ctx->tc_p2_lo, 4ull * Nb * ctx->tc_n2 * ctx->Ng_pad2)) != cudaSuccess)
        return bad(e, "tensor stage-2 operand (lo)");
    }
    // the retransform GEMM's matrix: BF16 (128-byte swizzle boxes), or hi +
    // lo BF16 for the split path (64-byte swizzle boxes)
    if (Nt <= 256) {
      auto upload = [&](bool transpose, void** hi_d, void** lo_d, CUtensorMap* tm, CUtensorMap* tm2,
                        CUtensorMap* tmp) -> cudaError_t {
        const std::vector<double> T = retransform_matrix(Nt, o.dt_mode, o.dt, transpose);
        std::vector<__nv_bfloat16> hi(T.size()), lo(T.size());
        for (size_t q = 0; q < T.size(); ++q) {
          hi[q] = __float2bfloat16_rn(static_cast<float>(T[q]));
          lo[q] = __float2bfloat16_rn(static_cast<float>(T[q] - static_cast<double>(__bfloat162float(hi[q]))));
        }
        const size_t tb = sizeof(__nv_bfloat16) * T.size();
        const int K = 2 * Nt, box = K > 256 ? 256 : K, bk = sp ? 32 : 64;
        cudaError_t r;
        if ((r = dalloc(hi_d, tb)) != cudaSuccess) return r;
        if ((r = cudaMemcpy(*hi_d, hi.data(), tb, cudaMemcpyHostToDevice)) != cudaSuccess) return r;
        if ((r = tc_encode_3d(tm, *hi_d, K, K, 1, K, box, bk)) != cudaSuccess) return r;
        if (!sp && (r = tc_encode_3d(tmp, *hi_d, K, K, 1, K, box / 2, bk)) != cudaSuccess) return r;
        if (sp) {
          if ((r = dalloc(lo_d, tb)) != cudaSuccess) return r;
          if ((r = cudaMemcpy(*lo_d, lo.data(), tb, cudaMemcpyHostToDevice)) != cudaSuccess) return r;
          if ((r = tc_encode_3d(tm2, *lo_d, K, K, 1, K, box, bk)) != cudaSuccess) return r;
        }
        return cudaSuccess;
      };
      if ((e = upload(false, &ctx->tc_T, &ctx->tc_T_lo, &ctx->tc_tmT, &ctx->tc_tmT2, &ctx->tc_tmTp)) != cudaSuccess)
        return bad(e, "retransform matrix");
      if (ctx->tc_adj &&
          (e = upload(true, &ctx->tc_Ta, &ctx->tc_Ta_lo, &ctx->tc_tmTa, &ctx->tc_tmTa2, &ctx->tc_tmTap)) != cudaSuccess)
        return bad(e, "adjoint retransform matrix");
    }
  }
  if ((e = launch_twiddles(ctx->tw, ctx->L, nullptr)) != cudaSuccess) return bad(e, "twiddles");
  if (ctx->df && (e = launch_twiddles_df(ctx->tw_df, ctx->L, nullptr)) != cudaSuccess) return bad(e, "pair twiddles");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bad(e, "create sync");
  *out = ctx;
  return S2W_OK;
}

int s2w_destroy(s2w_ctx* ctx) {
  if (!ctx) return S2W_OK;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return S2W_OK;
}

int s2w_operator_bytes(const s2w_ctx* ctx, size_t* g_bytes, size_t* p_bytes) {
  if (!ctx) return S2W_ERR_ARG;
  if (g_bytes) *g_bytes = ctx->g_bytes;
  if (p_bytes) *p_bytes = ctx->p_bytes;
  return S2W_OK;
}

namespace {

// Shared by the time-domain and the spectral loaders: spectra == true takes
// complex64 Ghat[l][r][j] ([Nb][ng][Ns]) instead of time-domain rows.
int load_greens_impl(s2w_ctx* ctx, int g0, int ng, const float* G, bool spectra, void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (!G || g0 < 0 || ng < 1 || static_cast<long long>(g0) + ng > ctx->Ng)
    return fail(ctx, S2W_ERR_ARG, "load_greens: rows [%d, %d) outside [0, %d) or G is NULL", g0, g0 + ng, ctx->Ng);
  const bool fp8 = ctx->opts.prec_g == S2W_PREC_FP8_E4M3;
  if (fp8 && (g0 % 256 != 0 || (ng % 256 != 0 && g0 + ng != ctx->Ng)))
    return fail(ctx, S2W_ERR_ARG, "load_greens: FP8 storage needs 256-row aligned chunks (g0=%d, ng=%d)", g0, ng);
  DeviceGuard guard(ctx->device);
  if (pointer_kind(G, ctx->device) < 0) return fail(ctx, S2W_ERR_ARG, "load_greens: G is on another device");
  if (ctx->fault == S2W_FAULT_OOM_LOAD)
    return fail(ctx, S2W_ERR_OOM, "load_greens: staging allocation failed (injected by the OOM_LOAD test hook)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long Ns = ctx->Ns, Nt = ctx->Nt, Nb = ctx->Nb, Ns_pad = ctx->Ns_pad;
  const long long RC = 256;
  float* stage_t = nullptr;
  float2* stage_s = nullptr;
  float2* stage_lo = nullptr;  // FP32_HILO: low-order parts of the spectra
  CK(cudaMalloc(&stage_t, sizeof(float) * RC * Ns * Nt));
  cudaError_t e = cudaMalloc(&stage_s, sizeof(float2) * Nb * RC * Ns_pad);
  if (e == cudaSuccess && ctx->df) e = cudaMalloc(&stage_lo, sizeof(float2) * Nb * RC * Ns_pad);
  if (e != cudaSuccess) {
    cudaFree(stage_t);
    cudaFree(stage_s);
    CK(e);
  }
  int rc_status = S2W_OK;
  for (long long r = 0; r < ng && rc_status == S2W_OK; r += RC) {
    const long long rc = std::min(RC, static_cast<long long>(ng) - r);
    const long long row0 = g0 + r;
    auto step = [&]() -> int {
      CK(cudaMemsetAsync(stage_s, 0, sizeof(float2) * Nb * rc * Ns_pad, st));
      // complex64 spectra carry no low-order part: lo = 0
      if (ctx->df) CK(cudaMemsetAsync(stage_lo, 0, sizeof(float2) * Nb * rc * Ns_pad, st));
      if (spectra) {  // bin l: rows r .. r+rc of Ghat_l, re-pitched to Ns_pad
        ctx->launches += fp8 ? 1 : 0;
        for (long long l = 0; l < Nb; ++l)
          CK(cudaMemcpy2DAsync(stage_s + l * rc * Ns_pad, sizeof(float2) * Ns_pad,
                               G + 2 * ((l * ng + r) * Ns), sizeof(float2) * Ns, sizeof(float2) * Ns, rc,
                               cudaMemcpyDefault, st));
      } else {
        CK(cudaMemcpyAsync(stage_t, G + r * Ns * Nt, sizeof(float) * rc * Ns * Nt, cudaMemcpyDefault, st));
        ctx->launches += fp8 ? 2 : 1;
        if (ctx->df)
          CK(launch_df_rfft_rows(stage_t, rc * Ns, static_cast<int>(Nt), static_cast<int>(ctx->L / 2), ctx->tw_df,
                                 stage_s, stage_lo, rc * Ns_pad, Ns, Ns_pad, st));
        else
          CK(launch_rfft_rows(stage_t, rc * Ns, static_cast<int>(Nt), static_cast<int>(ctx->L / 2), ctx->tw, stage_s,
                              rc * Ns_pad, Ns, Ns_pad, st));
      }
      ctx->launches += 1;
      if (ctx->df) {  // the pair's parts as two FP32 arrays of the same layout
        ctx->launches += 1;
        CK(launch_store_blocks(stage_s, static_cast<int>(Nb), rc * Ns_pad, EL_FP32, ctx->G, nullptr,
                               static_cast<long long>(ctx->Ng) * Ns_pad, row0 * Ns_pad, st));
        CK(launch_store_blocks(stage_lo, static_cast<int>(Nb), rc * Ns_pad, EL_FP32, ctx->G_lo, nullptr,
                               static_cast<long long>(ctx->Ng) * Ns_pad, row0 * Ns_pad, st));
      } else if (fp8) {
        CK(launch_fp8_store(stage_s, static_cast<int>(Nb), rc, static_cast<int>(Ns_pad), row0, ctx->Ng,
                            ctx->G_scale, ctx->nblk, ctx->G, st));
      } else {
        CK(launch_store_blocks(stage_s, static_cast<int>(Nb), rc * Ns_pad, ctx->opts.prec_g, ctx->G, ctx->G_lo,
                               static_cast<long long>(ctx->Ng) * Ns_pad, row0 * Ns_pad, st));
      }
      if (ctx->tc_adj) {  // Ghat_l^T[j][row0 + r] (transposing copy; grid along K)
        ctx->launches += 1;
        CK(launch_pack_a(stage_s, static_cast<int>(Nb), static_cast<int>(Ns), rc, rc * Ns_pad, 1, Ns_pad, Ns, 0, row0,
                         ctx->Ng_pad2, ctx->tc_gT, ctx->tc_gT_lo, st));
      }
      return S2W_OK;
    };
    rc_status = step();
  }
  if (rc_status == S2W_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc_status = fail(ctx, S2W_ERR_CUDA, "load_greens: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(st);
  cudaFree(stage_t);
  cudaFree(stage_s);
  cudaFree(stage_lo);
  if (rc_status != S2W_OK) return rc_status;
  for (int r = 0; r < ng; ++r) {
    if (!ctx->g_loaded[g0 + r]) ++ctx->g_count;
    ctx->g_loaded[g0 + r] = 1;
  }
  return S2W_OK;
}

// spectra == true takes complex64 Phat[l][o][r] ([Nb][No][ng]).
int load_adjoint_impl(s2w_ctx* ctx, int g0, int ng, const float* P, bool spectra, void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (!P || g0 < 0 || ng < 1 || static_cast<long long>(g0) + ng > ctx->Ng)
    return fail(ctx, S2W_ERR_ARG, "load_adjoint: columns [%d, %d) outside [0, %d) or P is NULL", g0, g0 + ng,
                ctx->Ng);
  DeviceGuard guard(ctx->device);
  if (pointer_kind(P, ctx->device) < 0) return fail(ctx, S2W_ERR_ARG, "load_adjoint: P is on another device");
  if (ctx->fault == S2W_FAULT_OOM_LOAD)
    return fail(ctx, S2W_ERR_OOM, "load_adjoint: staging allocation failed (injected by the OOM_LOAD test hook)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb;
  const long long RC = 2048;
  float* stage_t = nullptr;
  float2* stage_s = nullptr;
  float2* stage_lo = nullptr;  // FP32_HILO: low-order parts of the spectra
  CK(cudaMalloc(&stage_t, sizeof(float) * No * RC * Nt));
  cudaError_t e = cudaMalloc(&stage_s, sizeof(float2) * Nb * No * RC);
  if (e == cudaSuccess && ctx->df) e = cudaMalloc(&stage_lo, sizeof(float2) * Nb * No * RC);
  if (e != cudaSuccess) {
    cudaFree(stage_t);
    cudaFree(stage_s);
    CK(e);
  }
  int rc_status = S2W_OK;
  for (long long c = 0; c < ng && rc_status == S2W_OK; c += RC) {
    const long long rc = std::min(RC, static_cast<long long>(ng) - c);
    auto step = [&]() -> int {
      if (spectra) {  // bin l: columns c .. c+rc of every observation's row of Phat_l
        for (long long l = 0; l < Nb; ++l)
          CK(cudaMemcpy2DAsync(stage_s + l * No * rc, sizeof(float2) * rc, P + 2 * (l * No * ng + c),
                               sizeof(float2) * ng, sizeof(float2) * rc, No, cudaMemcpyDefault, st));
        // complex64 spectra carry no low-order part: lo = 0
        if (ctx->df) CK(cudaMemsetAsync(stage_lo, 0, sizeof(float2) * Nb * No * rc, st));
        ctx->launches += 1;
      } else {
        CK(cudaMemcpy2DAsync(stage_t, sizeof(float) * rc * Nt, P + c * Nt, sizeof(float) * ng * Nt,
                             sizeof(float) * rc * Nt, No, cudaMemcpyDefault, st));
        ctx->launches += 2;
        if (ctx->df)
          CK(launch_df_rfft_rows(stage_t, No * rc, static_cast<int>(Nt), static_cast<int>(ctx->L / 2), ctx->tw_df,
                                 stage_s, stage_lo, No * rc, rc, rc, st));
        else
          CK(launch_rfft_rows(stage_t, No * rc, static_cast<int>(Nt), static_cast<int>(ctx->L / 2), ctx->tw, stage_s,
                              No * rc, rc, rc, st));
      }
      if (ctx->single_pass && ctx->opts.dt_mode != S2W_DT_NONE) {  // fold D_t into the stage-2 spectra
        ctx->launches += 1;
        CK(launch_scale_dt(stage_s, static_cast<int>(Nb), No * rc, ctx->tw, static_cast<float>(1.0 / ctx->opts.dt),
                           st));
      }
      if (ctx->df) {  // the pair's parts as two FP32 arrays of the same layout
        ctx->launches += 1;
        CK(launch_store_adjoint(stage_s, static_cast<int>(Nb), static_cast<int>(No), rc, g0 + c, ctx->RL, ctx->nseg,
                                EL_FP32, ctx->P, st));
        CK(launch_store_adjoint(stage_lo, static_cast<int>(Nb), static_cast<int>(No), rc, g0 + c, ctx->RL,
                                ctx->nseg, EL_FP32, ctx->P_lo, st));
      } else {
        CK(launch_store_adjoint(stage_s, static_cast<int>(Nb), static_cast<int>(No), rc, g0 + c, ctx->RL, ctx->nseg,
                                ctx->opts.prec_p, ctx->P, st));
      }
      if (ctx->tc_on) {
        ctx->launches += 1;
        CK(launch_pack_b(stage_s, static_cast<int>(Nb), static_cast<int>(No), rc, No * rc, rc, g0 + c, ctx->Ng_pad2,
                         ctx->tc_p2h ? ctx->tc_n2 / 2 : ctx->tc_n2, ctx->tc_p2h ? 2 : 0, ctx->tc_p2, ctx->tc_p2_lo,
                         st));
      }
      if (ctx->tc_adj) {  // Phat_l^T[g0 + c + r][o] (transposing copy; observations along K)
        ctx->launches += 1;
        CK(launch_pack_a(stage_s, static_cast<int>(Nb), static_cast<int>(rc), No, No * rc, 1, rc, ctx->Ng, g0 + c, 0,
                         ctx->NoP, ctx->tc_pT, ctx->tc_pT_lo, st));
      }
      return S2W_OK;
    };
    rc_status = step();
  }
  if (rc_status == S2W_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc_status = fail(ctx, S2W_ERR_CUDA, "load_adjoint: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(st);
  cudaFree(stage_t);
  cudaFree(stage_s);
  cudaFree(stage_lo);
  if (rc_status != S2W_OK) return rc_status;
  for (int r = 0; r < ng; ++r) {
    if (!ctx->p_loaded[g0 + r]) ++ctx->p_count;
    ctx->p_loaded[g0 + r] = 1;
  }
  return S2W_OK;
}

}  // namespace

int s2w_load_greens(s2w_ctx* ctx, int g0, int ng, const float* G, void* stream) {
  return load_greens_impl(ctx, g0, ng, G, false, stream);
}

int s2w_load_greens_spectra(s2w_ctx* ctx, int g0, int ng, const float* Ghat, void* stream) {
  return load_greens_impl(ctx, g0, ng, Ghat, true, stream);
}

int s2w_load_adjoint(s2w_ctx* ctx, int g0, int ng, const float* P, void* stream) {
  return load_adjoint_impl(ctx, g0, ng, P, false, stream);
}

int s2w_load_adjoint_spectra(s2w_ctx* ctx, int g0, int ng, const float* Phat, void* stream) {
  return load_adjoint_impl(ctx, g0, ng, Phat, true, stream);
}

namespace {
// Tensor engine with host slip and host q, several sub-batches: sub-batch k's
// slip goes up on the copy stream while sub-batch k - 1 computes on `st`,
// and its waveforms come down while sub-batch k + 1 computes; the call
// returns when the last copy has landed.  Same kernels, launch shapes and
// results as the device-pointer path.
int waveforms_tensor_host(s2w_ctx* ctx, const float* slip, int B, float* q, cudaStream_t st) {
  const long long per_in = ctx->Ns * ctx->Nt, per_out = ctx->No * ctx->Nt;
  const int nsub = (B + ctx->tc_bsub - 1) / ctx->tc_bsub;
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  while (static_cast<int>(ctx->ev_in.size()) < nsub) {
    cudaEvent_t a, b;
    CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(a);
      return fail(ctx, S2W_ERR_CUDA, "waveforms: event creation failed");
    }
    ctx->ev_in.push_back(a);
    ctx->ev_out.push_back(b);
  }
  cudaStream_t cs = ctx->copy_stream;
  // the copy stream starts after the caller's earlier work (the workspaces)
  CK(cudaEventRecord(ctx->ev_out[0], st));
  CK(cudaStreamWaitEvent(cs, ctx->ev_out[0], 0));
  for (int k = 0; k < nsub; ++k) {
    const long long b0 = static_cast<long long>(k) * ctx->tc_bsub;
    const int Bs = static_cast<int>(std::min<long long>(ctx->tc_bsub, B - b0));
    CK(cudaMemcpyAsync(ctx->ws_slip + b0 * per_in, slip + b0 * per_in, sizeof(float) * Bs * per_in,
                       cudaMemcpyHostToDevice, cs));
    CK(cudaEventRecord(ctx->ev_in[k], cs));
  }
  const int* lens = ctx->cur_lens;
  int rc = S2W_OK;
  for (int k = 0; k < nsub && rc == S2W_OK; ++k) {
    const long long b0 = static_cast<long long>(k) * ctx->tc_bsub;
    const int Bs = static_cast<int>(std::min<long long>(ctx->tc_bsub, B - b0));
    CK(cudaStreamWaitEvent(st, ctx->ev_in[k], 0));
    ctx->cur_lens = lens ? lens + b0 : nullptr;
    rc = waveforms_tensor(ctx, ctx->ws_slip + b0 * per_in, Bs, ctx->ws_q + b0 * per_out, st);
    ctx->cur_lens = lens;
    if (rc != S2W_OK) break;
    CK(cudaEventRecord(ctx->ev_out[k], st));
    CK(cudaStreamWaitEvent(cs, ctx->ev_out[k], 0));
    CK(cudaMemcpyAsync(q + b0 * per_out, ctx->ws_q + b0 * per_out, sizeof(float) * Bs * per_out,
                       cudaMemcpyDeviceToHost, cs));
  }
  // the caller's stream continues after the copies (workspace reuse), and
  // the host after the last one
  CK(cudaEventRecord(ctx->ev_in[0], cs));
  CK(cudaStreamWaitEvent(st, ctx->ev_in[0], 0));
  CK(cudaStreamSynchronize(cs));
  return rc;
}
}  // namespace

int s2w_waveforms(s2w_ctx* ctx, const float* slip, int B, float* q, float* seafloor, void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (B < 0 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "waveforms: B=%d outside [0, max_batch=%d]", B, ctx->opts.max_batch);
  if (B == 0) return S2W_OK;
  if (!slip || !q) return fail(ctx, S2W_ERR_ARG, "waveforms: slip and q must not be NULL");
  if (ctx->g_count != ctx->Ng || ctx->p_count != ctx->Ng)
    return fail(ctx, S2W_ERR_STATE, "waveforms: operators not fully loaded (%lld/%d Green rows, %lld/%d adjoint cols)",
                ctx->g_count, ctx->Ng, ctx->p_count, ctx->Ng);
  DeviceGuard guard(ctx->device);
  const int ks = pointer_kind(slip, ctx->device), kq = pointer_kind(q, ctx->device);
  const int kf = seafloor ? pointer_kind(seafloor, ctx->device) : 1;
  if (ks < 0 || kq < 0 || kf < 0) return fail(ctx, S2W_ERR_ARG, "waveforms: pointer on another device");
  if (ctx->fault == S2W_FAULT_LAUNCH)
    return fail(ctx, S2W_ERR_CUDA, "waveforms: kernel launch failed (injected by the LAUNCH test hook)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long Ns = ctx->Ns, Ng = ctx->Ng, No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb, Ns_pad = ctx->Ns_pad;
  if (ctx->single_pass && seafloor != nullptr)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "waveforms: no seafloor output in the single-pass variant");
  const bool use_tc = ctx->tc_on && seafloor == nullptr && (ctx->tc_split || ctx->tc_T != nullptr) &&
                      (ctx->opts.engine == S2W_ENGINE_TENSOR || B >= ctx->tc_min_batch);
  if (use_tc && ks == 0 && kq == 0 && B > ctx->tc_bsub) return waveforms_tensor_host(ctx, slip, B, q, st);
  const float* slip_d = slip;
  if (ks == 0) {
    StageTimer t(ctx, 5, st, 0);
    CK(cudaMemcpyAsync(ctx->ws_slip, slip, sizeof(float) * B * Ns * Nt, cudaMemcpyHostToDevice, st));
    slip_d = ctx->ws_slip;
  }
  float* q_d = kq == 1 ? q : ctx->ws_q;
  if (use_tc) {
    int rc = waveforms_tensor(ctx, slip_d, B, q_d, st);
    if (rc != S2W_OK) return rc;
    if (kq == 0) {
      StageTimer t(ctx, 5, st, 0);
      CK(cudaMemcpyAsync(q, q_d, sizeof(float) * B * No * Nt, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    return S2W_OK;
  }
  for (int g0 = 0; g0 < B; g0 += kStreamGroup) {
    const int Bg = std::min(kStreamGroup, B - g0);
    // K1
    {
      StageTimer t(ctx, 0, st);
      if (ctx->df)
        CK(launch_df_rfft_rows(slip_d + static_cast<long long>(g0) * Ns * Nt, Bg * Ns, static_cast<int>(Nt),
                               static_cast<int>(ctx->L / 2), ctx->tw_df, ctx->ws_shat, ctx->ws_shat_lo, Bg * Ns_pad,
                               Ns, Ns_pad, st, ctx->cur_lens ? ctx->cur_lens + g0 : nullptr));
      else
        CK(launch_rfft_rows(slip_d + static_cast<long long>(g0) * Ns * Nt, Bg * Ns, static_cast<int>(Nt),
                            static_cast<int>(ctx->L / 2), ctx->tw, ctx->ws_shat, Bg * Ns_pad, Ns, Ns_pad, st,
                            ctx->cur_lens ? ctx->cur_lens + g0 : nullptr));
    }
    const long long part_b = Nb * ctx->nseg * No;
    for (int b = 0; b < Bg; ++b) {
      const long long bg = g0 + b;  // rupture index in the call
      // K2
      StreamArgs a1{};
      a1.rows = ctx->G;
      a1.rows_lo = ctx->G_lo;
      a1.F = Nb * Ng;
      a1.row_len = static_cast<int>(Ns_pad);
      a1.el = ctx->opts.prec_g;
      a1.x = ctx->ws_shat + b * Ns_pad;
      a1.x_stride = Bg * Ns_pad;
      a1.rows_per_vec = Ng;
      a1.scale = ctx->G_scale;
      a1.nblk = ctx->nblk;
      a1.y = ctx->ws_mhat;
      if (ctx->df) {
        a1.x_lo = ctx->ws_shat_lo + b * Ns_pad;
        a1.y_lo = ctx->ws_mhat_lo;
      }
      a1.status = ctx->d_status;
      a1.wait_ns = ctx->wait_ns;
      a1.fault_skip = ctx->fault == S2W_FAULT_WAIT ? 1 : 0;
      {
        StageTimer t(ctx, 1, st);
        CK(launch_stream_dot(a1, ctx->num_sms, st));
      }
      // K3
      float* sf = nullptr;
      if (seafloor) sf = kf == 1 ? seafloor + bg * Ng * Nt : ctx->ws_seafloor;
      if (ctx->single_pass) {  // mhat goes to stage 2 as it is, in the segment layout
        StageTimer t(ctx, 2, st, 0);
        CK(cudaMemcpy2DAsync(ctx->ws_vhat, sizeof(float2) * ctx->nseg * ctx->RL, ctx->ws_mhat, sizeof(float2) * Ng,
                             sizeof(float2) * Ng, Nb, cudaMemcpyDeviceToDevice, st));
      } else if (ctx->df) {
        StageTimer t(ctx, 2, st);
        CK(launch_df_retransform(ctx->ws_mhat, ctx->ws_mhat_lo, Ng, Ng, static_cast<int>(Nt), ctx->tw_df,
                                 1.0 / ctx->opts.dt, ctx->opts.dt_mode, ctx->ws_vhat, ctx->ws_vhat_lo,
                                 static_cast<long long>(ctx->nseg) * ctx->RL, sf, st));
      } else {
        StageTimer t(ctx, 2, st);
        CK(launch_retransform(ctx->ws_mhat, Ng, Ng, static_cast<int>(Nt), ctx->tw,
                              static_cast<float>(1.0 / ctx->opts.dt), ctx->opts.dt_mode, ctx->ws_vhat,
                              static_cast<long long>(ctx->nseg) * ctx->RL, sf, st));
      }
      if (seafloor && kf == 0)
        CK(cudaMemcpyAsync(seafloor + bg * Ng * Nt, ctx->ws_seafloor, sizeof(float) * Ng * Nt,
                           cudaMemcpyDeviceToHost, st));
      // K4
      StreamArgs a2{};
      a2.rows = ctx->P;
      a2.F = Nb * ctx->nseg * No;
      a2.row_len = ctx->RL;
      a2.el = ctx->opts.prec_p;
      a2.x = ctx->ws_vhat;
      a2.x_stride = ctx->RL;
      a2.rows_per_vec = No;
      a2.y = ctx->ws_part + b * part_b;
      if (ctx->df) {
        a2.rows_lo = ctx->P_lo;
        a2.x_lo = ctx->ws_vhat_lo;
        a2.y_lo = ctx->ws_part_lo + b * part_b;
      }
      a2.status = ctx->d_status;
      a2.wait_ns = ctx->wait_ns;
      {
        StageTimer t(ctx, 3, st);
        CK(launch_stream_dot(a2, ctx->num_sms, st));
      }
    }
    // K5
    {
      StageTimer t(ctx, 4, st);
      if (ctx->df)
        CK(launch_df_reduce_irfft(ctx->ws_part, ctx->ws_part_lo, Bg, static_cast<int>(No), ctx->nseg,
                                  static_cast<int>(ctx->L / 2), part_b, static_cast<long long>(ctx->nseg) * No, No,
                                  ctx->tw_df, q_d + static_cast<long long>(g0) * No * Nt, st, static_cast<int>(Nt)));
      else
        CK(launch_reduce_irfft(ctx->ws_part, Bg, static_cast<int>(No), ctx->nseg, static_cast<int>(ctx->L / 2),
                               part_b, static_cast<long long>(ctx->nseg) * No, No, ctx->tw,
                               q_d + static_cast<long long>(g0) * No * Nt, st, static_cast<int>(Nt)));
    }
  }
  if (kq == 0) {
    StageTimer t(ctx, 5, st, 0);
    CK(cudaMemcpyAsync(q, q_d, sizeof(float) * B * No * Nt, cudaMemcpyDeviceToHost, st));
  }
  if (kq == 0 || (seafloor && kf == 0)) CK(cudaStreamSynchronize(st));
  return S2W_OK;
}

int s2w_waveforms_active(s2w_ctx* ctx, const float* slip, const int* active_len, int B, float* q, float* seafloor,
                         void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (B < 0 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "waveforms_active: B=%d outside [0, max_batch=%d]", B, ctx->opts.max_batch);
  if (B == 0) return S2W_OK;
  if (!active_len) return s2w_waveforms(ctx, slip, B, q, seafloor, stream);
  DeviceGuard guard(ctx->device);
  if (pointer_kind(active_len, ctx->device) != 0)
    return fail(ctx, S2W_ERR_ARG, "waveforms_active: active_len must be a host array");
  for (int b = 0; b < B; ++b)
    if (active_len[b] < 0 || active_len[b] > ctx->Nt)
      return fail(ctx, S2W_ERR_ARG, "waveforms_active: active_len[%d] = %d outside [0, Nt=%lld]", b, active_len[b],
                  ctx->Nt);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(ctx->ws_lens, active_len, sizeof(int) * B, cudaMemcpyHostToDevice, st));
  ctx->cur_lens = ctx->ws_lens;
  const int rc = s2w_waveforms(ctx, slip, B, q, seafloor, stream);
  ctx->cur_lens = nullptr;
  return rc;
}

int s2w_adjoint(s2w_ctx* ctx, const float* r, int B, float* grad_s, void* stream) {
  if (ctx && ctx->single_pass)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "adjoint: not available in the single-pass variant");
  if (ctx && ctx->df) return fail(ctx, S2W_ERR_UNSUPPORTED, "adjoint: not available with FP32_HILO storage");
  if (!ctx) return S2W_ERR_ARG;
  if (B < 0 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "adjoint: B=%d outside [0, max_batch=%d]", B, ctx->opts.max_batch);
  if (B == 0) return S2W_OK;
  if (!r || !grad_s) return fail(ctx, S2W_ERR_ARG, "adjoint: r and grad_s must not be NULL");
  if (ctx->g_count != ctx->Ng || ctx->p_count != ctx->Ng)
    return fail(ctx, S2W_ERR_STATE, "adjoint: operators not fully loaded");
  DeviceGuard guard(ctx->device);
  const int kr = pointer_kind(r, ctx->device), kg = pointer_kind(grad_s, ctx->device);
  if (kr < 0 || kg < 0) return fail(ctx, S2W_ERR_ARG, "adjoint: pointer on another device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long Ns = ctx->Ns, Ng = ctx->Ng, No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb, Ns_pad = ctx->Ns_pad;
  const float* r_d = r;
  if (kr == 0) {
    StageTimer t(ctx, 5, st, 0);
    CK(cudaMemcpyAsync(ctx->ws_q, r, sizeof(float) * B * No * Nt, cudaMemcpyHostToDevice, st));
    r_d = ctx->ws_q;
  }
  float* g_d = kg == 1 ? grad_s : ctx->ws_slip;
  if (ctx->tc_adj && (ctx->opts.engine == S2W_ENGINE_TENSOR || B >= ctx->tc_min_batch)) {
    const int rc = adjoint_tensor(ctx, r_d, B, g_d, st);
    if (rc != S2W_OK) return rc;
    if (kg == 0) {
      StageTimer t(ctx, 5, st, 0);
      CK(cudaMemcpyAsync(grad_s, g_d, sizeof(float) * B * Ns * Nt, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    return S2W_OK;
  }
  {
    StageTimer t(ctx, 0, st);
    CK(launch_rfft_rows(r_d, B * No, static_cast<int>(Nt), static_cast<int>(Nt), ctx->tw, ctx->ws_rhat, B * No, No,
                        No, st));
  }
  const int dt_t = ctx->opts.dt_mode == S2W_DT_NONE ? S2W_DT_NONE : kDtTranspose;
  for (int b = 0; b < B; ++b) {
    {  // stage-2 adjoint: what_l[i] = sum_o conj(Phat_l[o][i]) rhat_l[o]
      StageTimer t(ctx, 3, st);
      StreamTArgs a{};
      a.rows = ctx->P;
      a.el = ctx->opts.prec_p;
      a.row_len = ctx->RL;
      a.n_units = Nb * ctx->nseg;
      a.G1 = No;
      a.Rc = static_cast<int>(No);
      a.nchunk = 1;
      a.w = ctx->ws_rhat;
      a.w_base = static_cast<long long>(b) * No;
      a.wa = ctx->nseg;
      a.wb = static_cast<long long>(B) * No;
      a.y = ctx->ws_vhat;
      a.status = ctx->d_status;
      CK(launch_stream_tdot(a, ctx->num_sms, st));
    }
    {  // IFFT + Truncate, D_t^T, ZeroPad + FFT
      StageTimer t(ctx, 2, st);
      CK(launch_retransform(ctx->ws_vhat, Ng, static_cast<long long>(ctx->nseg) * ctx->RL, static_cast<int>(Nt),
                            ctx->tw, static_cast<float>(1.0 / ctx->opts.dt), dt_t, ctx->ws_mhat, Ng, nullptr, st));
    }
    {  // stage-1 adjoint: ghat_l[j] = sum_i conj(Ghat_l[i][j]) uhat_l[i], in row chunks
      StageTimer t(ctx, 1, st);
      StreamTArgs a{};
      a.rows = ctx->G;
      a.rows_lo = ctx->G_lo;
      a.el = ctx->opts.prec_g;
      a.row_len = static_cast<int>(Ns_pad);
      a.n_units = Nb * ctx->adj_nchunk;
      a.G1 = Ng;
      a.Rc = ctx->adj_rc;
      a.nchunk = ctx->adj_nchunk;
      a.w = ctx->ws_mhat;
      a.w_base = 0;
      a.wa = 1;
      a.wb = Ng;
      a.scale = ctx->G_scale;
      a.nblk = ctx->nblk;
      a.y = ctx->ws_gpart;
      a.status = ctx->d_status;
      CK(launch_stream_tdot(a, ctx->num_sms, st));
    }
    {  // chunk reduction + IFFT + Truncate -> grad_s[b]
      StageTimer t(ctx, 4, st);
      CK(launch_reduce_irfft(ctx->ws_gpart, 1, static_cast<int>(Ns), ctx->adj_nchunk, static_cast<int>(Nt), 0,
                             static_cast<long long>(ctx->adj_nchunk) * Ns_pad, Ns_pad, ctx->tw,
                             g_d + static_cast<long long>(b) * Ns * Nt, st));
    }
  }
  if (kg == 0) {
    StageTimer t(ctx, 5, st, 0);
    CK(cudaMemcpyAsync(grad_s, g_d, sizeof(float) * B * Ns * Nt, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return S2W_OK;
}

int s2w_misfit_gradient(s2w_ctx* ctx, const float* slip, const float* d, int B, float* grad_s, float* loss,
                        void* stream) {
  if (ctx && ctx->single_pass)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "misfit_gradient: not available in the single-pass variant");
  if (ctx && ctx->df) return fail(ctx, S2W_ERR_UNSUPPORTED, "misfit_gradient: not available with FP32_HILO storage");
  if (!ctx) return S2W_ERR_ARG;
  if (B < 0 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "misfit_gradient: B=%d outside [0, max_batch=%d]", B, ctx->opts.max_batch);
  if (B == 0) return S2W_OK;
  if (!slip || !d || !grad_s) return fail(ctx, S2W_ERR_ARG, "misfit_gradient: slip, d, grad_s must not be NULL");
  DeviceGuard guard(ctx->device);
  const int kd = pointer_kind(d, ctx->device), kg = pointer_kind(grad_s, ctx->device);
  const int kl = loss ? pointer_kind(loss, ctx->device) : kg;
  if (kd < 0 || kg < 0 || kl < 0) return fail(ctx, S2W_ERR_ARG, "misfit_gradient: pointer on another device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n_per_b = static_cast<long long>(ctx->No) * ctx->Nt;
  int rc = s2w_waveforms(ctx, slip, B, ctx->ws_resid, nullptr, stream);
  if (rc != S2W_OK) return rc;
  const float* d_d = d;
  if (kd == 0) {
    StageTimer t(ctx, 5, st, 0);
    CK(cudaMemcpyAsync(ctx->ws_d, d, sizeof(float) * B * n_per_b, cudaMemcpyHostToDevice, st));
    d_d = ctx->ws_d;
  }
  {
    StageTimer t(ctx, 4, st);
    CK(launch_residual(ctx->ws_resid, d_d, B, n_per_b, loss && kl == 1 ? loss : ctx->ws_loss, st));
  }
  rc = s2w_adjoint(ctx, ctx->ws_resid, B, grad_s, stream);
  if (rc != S2W_OK) return rc;
  if (loss && kl == 0) {
    CK(cudaMemcpyAsync(loss, ctx->ws_loss, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return S2W_OK;
}

int s2w_rfft(s2w_ctx* ctx, const float* x, long long rows, float* X, void* stream) {
  if (ctx && ctx->single_pass)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "rfft: not available in the single-pass variant");
  if (!ctx) return S2W_ERR_ARG;
  if (rows < 0 || (rows > 0 && (!x || !X))) return fail(ctx, S2W_ERR_ARG, "rfft: bad arguments");
  if (rows == 0) return S2W_OK;
  DeviceGuard guard(ctx->device);
  if (pointer_kind(x, ctx->device) != 1 || pointer_kind(X, ctx->device) != 1)
    return fail(ctx, S2W_ERR_ARG, "rfft: x and X must be device pointers");
  ctx->launches += 1;
  CK(launch_rfft_rows(x, rows, ctx->Nt, ctx->Nt, ctx->tw, reinterpret_cast<float2*>(X), 1, 1, ctx->Nb,
                      static_cast<cudaStream_t>(stream)));
  return S2W_OK;
}

int s2w_irfft(s2w_ctx* ctx, const float* X, long long rows, float* x, void* stream) {
  if (ctx && ctx->single_pass)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "irfft: not available in the single-pass variant");
  if (!ctx) return S2W_ERR_ARG;
  if (rows < 0 || (rows > 0 && (!x || !X))) return fail(ctx, S2W_ERR_ARG, "irfft: bad arguments");
  if (rows == 0) return S2W_OK;
  DeviceGuard guard(ctx->device);
  if (pointer_kind(x, ctx->device) != 1 || pointer_kind(X, ctx->device) != 1)
    return fail(ctx, S2W_ERR_ARG, "irfft: x and X must be device pointers");
  ctx->launches += 1;
  CK(launch_irfft_rows(reinterpret_cast<const float2*>(X), rows, ctx->Nt, ctx->tw, x,
                       static_cast<cudaStream_t>(stream)));
  return S2W_OK;
}

// Graphs kept per context; a call with a new (slip, q, B) beyond this evicts
// the least recently replayed one.
constexpr size_t kGraphCache = 8;

int s2w_waveforms_graph(s2w_ctx* ctx, const float* slip, int B, float* q, void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (B < 0 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "waveforms_graph: B=%d outside [0, max_batch=%d]", B, ctx->opts.max_batch);
  if (B == 0) return S2W_OK;
  if (!slip || !q) return fail(ctx, S2W_ERR_ARG, "waveforms_graph: slip and q must not be NULL");
  if (ctx->g_count != ctx->Ng || ctx->p_count != ctx->Ng)
    return fail(ctx, S2W_ERR_STATE, "waveforms_graph: operators not fully loaded");
  DeviceGuard guard(ctx->device);
  if (pointer_kind(slip, ctx->device) != 1 || pointer_kind(q, ctx->device) != 1)
    return fail(ctx, S2W_ERR_ARG, "waveforms_graph: slip and q must be device pointers of the context's device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s2w_ctx::GraphEntry* ge = nullptr;
  for (auto& g : ctx->graphs)
    if (g.slip == slip && g.q == q && g.B == B) ge = &g;
  if (ge == nullptr) {
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    // the captured work must come after earlier work on `stream` (operators
    // loaded, inputs written): capture happens on a separate stream
    CK(cudaStreamSynchronize(st));
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;
    const long long l0 = ctx->launches;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
    const int rc = s2w_waveforms(ctx, slip, B, q, nullptr, ctx->cap_stream);
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->prof_on = prof;
    const long long n_launch = ctx->launches - l0;
    ctx->launches = l0;
    if (rc != S2W_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CK(ec);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    if (ctx->graphs.size() >= kGraphCache) {
      size_t old = 0;
      for (size_t k = 1; k < ctx->graphs.size(); ++k)
        if (ctx->graphs[k].last_use < ctx->graphs[old].last_use) old = k;
      cudaGraphExecDestroy(ctx->graphs[old].exec);
      ctx->graphs.erase(ctx->graphs.begin() + static_cast<long>(old));
    }
    ctx->graphs.push_back({slip, q, B, exec, n_launch, 0});
    ge = &ctx->graphs.back();
  }
  ge->last_use = ++ctx->graph_clock;
  StageTimer t(ctx, 7, st, static_cast<int>(ge->launches));
  CK(cudaGraphLaunch(ge->exec, st));
  return S2W_OK;
}

}  // extern "C"

namespace {

// Autotuner cache: one text line per problem,
//   s2w-tune-1 <key> bsub=<n> pair=<n> s2c=<n> minb=<n>
// with <key> naming everything the choices depend on.  A later entry for the
// same key replaces the earlier one.
std::string tune_key(const s2w_ctx* ctx, int B) {
  cudaDeviceProp pr;
  char name[256] = "unknown";
  if (cudaGetDeviceProperties(&pr, ctx->device) == cudaSuccess) {
    std::snprintf(name, sizeof(name), "%s", pr.name);
    for (char* c = name; *c; ++c)
      if (*c == ' ' || *c == '\t') *c = '_';
  }
  char k[512];
  std::snprintf(k, sizeof(k), "Ns=%d,Ng=%d,No=%d,Nt=%d,B=%d,pg=%d,pp=%d,f8a=%d,adj=%d,bmax=%d,sms=%d,gpu=%s", ctx->Ns,
                ctx->Ng, ctx->No, ctx->Nt, B, ctx->opts.prec_g, ctx->opts.prec_p, ctx->opts.tc_fp8_act,
                ctx->opts.tc_adjoint, ctx->tc_bsub_max, ctx->num_sms, name);
  return k;
}

bool tune_cache_read(const std::string& path, const std::string& key, int* bsub, int* pair, int* s2c, int* minb) {
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char k[600];
    int b, p, c, m;
    if (std::sscanf(line, "s2w-tune-1 %599s bsub=%d pair=%d s2c=%d minb=%d", k, &b, &p, &c, &m) == 5 && key == k) {
      *bsub = b;
      *pair = p;
      *s2c = c;
      *minb = m;
      found = true;  // keep reading: the last entry for the key wins
    }
  }
  std::fclose(f);
  return found;
}

// Rewrites the file with the entry for `key` replaced (written to a temporary
// file next to it, then renamed over it).
bool tune_cache_write(const std::string& path, const std::string& key, int bsub, int pair, int s2c, int minb) {
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path.c_str(), "r")) {
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
      char k[600];
      if (std::sscanf(line, "s2w-tune-1 %599s", k) == 1 && key == k) continue;
      keep.emplace_back(line);
    }
    std::fclose(f);
  }
  char tmp_name[64];
  std::snprintf(tmp_name, sizeof(tmp_name), ".tmp%d", static_cast<int>(std::rand() & 0xffffff));
  const std::string tmp = path + tmp_name;
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  for (const auto& l : keep) std::fputs(l.c_str(), f);
  std::fprintf(f, "s2w-tune-1 %s bsub=%d pair=%d s2c=%d minb=%d\n", key.c_str(), bsub, pair, s2c, minb);
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

// GEMM-form knob of the tensor engine: the public S2W_PAIR_* value and the
// internal tc_pair code it selects.
int pair_code(int pub) { return pub == S2W_PAIR_ON ? 1 : (pub == S2W_PAIR_OFF ? 0 : kDefaultPair); }
// The GEMM form of a public pair value: S2W_PAIR_ON also runs the BF16
// retransform GEMM on two-SM tiles, as when the caller sets it.
void apply_pair_mode(s2w_ctx* ctx, int pub) {
  ctx->tc_pair = pair_code(pub);
  ctx->tc_rtpair = pub == S2W_PAIR_ON;
}

}  // namespace

extern "C" {

int s2w_autotune(s2w_ctx* ctx, int B, s2w_tuning* out, void* stream) {
  if (!ctx) return S2W_ERR_ARG;
  if (B < 1 || B > ctx->opts.max_batch)
    return fail(ctx, S2W_ERR_ARG, "autotune: B=%d outside [1, max_batch=%d]", B, ctx->opts.max_batch);
  if (ctx->g_count != ctx->Ng || ctx->p_count != ctx->Ng)
    return fail(ctx, S2W_ERR_STATE, "autotune: operators not fully loaded");
  DeviceGuard guard(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // captured graphs hold the old schedule
  CK(cudaStreamSynchronize(st));
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  s2w_tuning r{};
  const bool tensor = ctx->tc_on && (ctx->tc_split || ctx->tc_T != nullptr);
  const std::string key = tune_key(ctx, B);
  // the public pair value of the current form (AUTO unless the caller fixed one)
  int pair_pub = ctx->opts.tc_pair;
  if (tensor && !ctx->tune_cache.empty()) {
    int b = 0, p = 0, c = 0, m = 0;
    if (tune_cache_read(ctx->tune_cache, key, &b, &p, &c, &m) && b >= 1 && b <= ctx->tc_bsub_max &&
        (p == S2W_PAIR_AUTO || p == S2W_PAIR_ON || p == S2W_PAIR_OFF) && c >= 1 && c <= ctx->s2_max_chunks &&
        m >= 1) {
      ctx->tc_bsub = b;
      apply_pair_mode(ctx, p);
      set_s2_chunks(ctx, c);
      ctx->tc_min_batch = m;
      r.from_cache = 1;
      r.tc_bsub = ctx->tc_bsub;
      r.tc_pair = p;
      r.tc_s2_chunks = ctx->tc_nkc;
      r.tc_min_batch = m;
      if (out) *out = r;
      return S2W_OK;
    }
  }
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  const long long l0 = ctx->launches;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // dummy inputs: the slip workspace (any values; the timings do not depend on them)
  auto timed = [&](int nb, int engine, float* ms) -> int {
    const int saved = ctx->opts.engine;
    ctx->opts.engine = engine;
    int rc = s2w_waveforms(ctx, ctx->ws_slip, nb, ctx->ws_q, nullptr, st);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 2 && rc == S2W_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = s2w_waveforms(ctx, ctx->ws_slip, nb, ctx->ws_q, nullptr, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float m = 0.f;
      cudaEventElapsedTime(&m, e0, e1);
      best = std::min(best, m);
    }
    ctx->opts.engine = saved;
    *ms = best;
    return rc;
  };
  int rc = timed(1, S2W_ENGINE_STREAM, &r.ms_stream_per_rupture);
  r.tc_min_batch = ctx->tc_min_batch;
  r.tc_bsub = ctx->tc_bsub;
  r.tc_pair = pair_pub;
  r.tc_s2_chunks = ctx->tc_nkc;
  if (rc == S2W_OK && tensor) {
    r.probe_batch = std::min(B, ctx->tc_bsub_max);
    // 1. the GEMM form: ruptures per pass x pair mode (fixed options are not searched)
    // (the 128-rupture passes only when the probe batch needs two of them)
    const int bsubs[2] = {ctx->tc_bsub_max, ctx->tc_bsub_max > 128 && r.probe_batch > 128 ? 128 : 0};
    const int pairs[3] = {S2W_PAIR_AUTO, S2W_PAIR_OFF, S2W_PAIR_ON};
    float best = 1e30f;
    int best_b = ctx->tc_bsub, best_p = pair_pub, nf = 0;
    for (int i = 0; i < 2 && rc == S2W_OK; ++i) {
      if (bsubs[i] == 0 || (ctx->opts.tc_bsub != 0 && bsubs[i] != ctx->opts.tc_bsub)) continue;
      for (int j = 0; j < 3 && rc == S2W_OK; ++j) {
        if (ctx->opts.tc_pair != S2W_PAIR_AUTO && pairs[j] != ctx->opts.tc_pair) continue;
        ctx->tc_bsub = bsubs[i];
        apply_pair_mode(ctx, pairs[j]);
        set_s2_chunks(ctx, ctx->opts.tc_s2_chunks);
        r.form_bsub[nf] = bsubs[i];
        r.form_pair[nf] = pairs[j];
        rc = timed(r.probe_batch, S2W_ENGINE_TENSOR, &r.ms_form[nf]);
        if (rc == S2W_OK && r.ms_form[nf] < best) {
          best = r.ms_form[nf];
          best_b = bsubs[i];
          best_p = pairs[j];
        }
        ++nf;
      }
    }
    ctx->tc_bsub = best_b;
    apply_pair_mode(ctx, best_p);
    set_s2_chunks(ctx, ctx->opts.tc_s2_chunks);
    r.tc_bsub = best_b;
    r.tc_pair = best_p;
    // 2. the stage-2 K chunk count around the round-balance choice.  The
    // split precision tries no count below it (it starts at the chunk
    // length kSplitChunkK: see there)
    int best_c = ctx->tc_nkc;
    if (rc == S2W_OK && ctx->opts.tc_s2_chunks == 0) {
      const int h = ctx->tc_nkc;
      const bool longer_ok = !ctx->tc_split;
      const int cand[4] = {h, longer_ok ? std::max(1, h / 2) : h, std::min(ctx->s2_max_chunks, 2 * h),
                           longer_ok ? 1 : h};
      float best_s2 = 1e30f;
      for (int k = 0; k < 4 && rc == S2W_OK; ++k) {
        bool dup = false;
        for (int j = 0; j < k; ++j) dup = dup || r.s2_chunk_cand[j] == cand[k];
        if (dup) continue;
        set_s2_chunks(ctx, cand[k]);
        r.s2_chunk_cand[k] = ctx->tc_nkc;
        rc = timed(r.probe_batch, S2W_ENGINE_TENSOR, &r.ms_s2_chunks[k]);
        if (rc == S2W_OK && r.ms_s2_chunks[k] < best_s2) {
          best_s2 = r.ms_s2_chunks[k];
          best_c = ctx->tc_nkc;
        }
      }
      set_s2_chunks(ctx, best_c);
    }
    r.tc_s2_chunks = ctx->tc_nkc;
    // 3. the smallest batch whose tensor pass beats that many stream passes
    const int sizes[7] = {1, 2, 4, 8, 16, 32, 64};
    int min_b = 0;
    for (int k = 0; k < 7 && rc == S2W_OK; ++k) {
      if (sizes[k] > B || sizes[k] > ctx->tc_bsub) break;
      rc = timed(sizes[k], S2W_ENGINE_TENSOR, &r.ms_tensor_batch[k]);
      if (rc == S2W_OK && min_b == 0 && r.ms_tensor_batch[k] < sizes[k] * r.ms_stream_per_rupture) min_b = sizes[k];
    }
    if (min_b == 0) min_b = r.ms_tensor_batch[0] > 0.f ? ctx->tc_bsub + 1 : ctx->tc_min_batch;
    ctx->tc_min_batch = min_b;
    r.tc_min_batch = min_b;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->prof_on = prof;
  ctx->launches = l0;
  if (rc != S2W_OK) return rc;
  if (tensor && !ctx->tune_cache.empty() &&
      !tune_cache_write(ctx->tune_cache, key, r.tc_bsub, r.tc_pair, r.tc_s2_chunks, r.tc_min_batch))
    return fail(ctx, S2W_ERR_ARG, "autotune: cannot write the cache file %s", ctx->tune_cache.c_str());
  if (out) *out = r;
  return S2W_OK;
}

int s2w_profile_enable(s2w_ctx* ctx, int on) {
  if (!ctx) return S2W_ERR_ARG;
  DeviceGuard guard(ctx->device);
  for (auto& p : ctx->pending) {
    cudaEventSynchronize(p.b);
    ctx->ev_free.push_back(p.a);
    ctx->ev_free.push_back(p.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < S2W_NUM_STAGES; ++i) {
    ctx->prof_ms[i] = 0.0;
    ctx->prof_cnt[i] = 0;
  }
  ctx->prof_on = on != 0;
  return S2W_OK;
}

int s2w_profile_read(s2w_ctx* ctx, s2w_profile* out) {
  if (!ctx || !out) return S2W_ERR_ARG;
  DeviceGuard guard(ctx->device);
  for (auto& p : ctx->pending) {
    CK(cudaEventSynchronize(p.b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    ctx->prof_ms[p.stage] += ms;
    ctx->prof_cnt[p.stage] += 1;
    ctx->ev_free.push_back(p.a);
    ctx->ev_free.push_back(p.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < S2W_NUM_STAGES; ++i) {
    out->ms[i] = ctx->prof_ms[i];
    out->count[i] = ctx->prof_cnt[i];
  }
  out->launches = ctx->launches;
  return S2W_OK;
}

int s2w_sync(s2w_ctx* ctx) {
  if (!ctx) return S2W_ERR_ARG;
  DeviceGuard guard(ctx->device);
  CK(cudaDeviceSynchronize());
  int h = 0;
  CK(cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
    return fail(ctx, S2W_ERR_TIMEOUT, "a kernel-side wait expired (status bits 0x%x)", h);
  }
  return S2W_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Waveforms without allocating: scratch in a fixed static device array.
//
// s2w_waveforms keeps its intermediates (slip spectra, seafloor spectra,
// velocity spectra, stage-2 partials) in workspaces that s2w_create allocates.
// Some callers cannot let a library allocate device memory on their behalf:
// a host application whose device memory all comes from its own pool, code
// that runs inside a CUDA stream capture (where a cudaMalloc would break the
// capture), or a latency-bound warning loop that must never wait on the
// allocator.  s2w_waveforms_noalloc evaluates one rupture with the same
// kernels but takes every intermediate from kNoAllocScratchBytes of static
// device memory, so the call itself allocates nothing.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// Every GPU that loads libs2w holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Device address of g_noalloc_scratch on the current device (== `device`).
// The symbol's name in host code is only a host-side stand-in; the real
// address comes from cudaGetSymbolAddress, taken once per device.
int noalloc_scratch(s2w_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "waveforms_noalloc: device ordinal %d", ctx->device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[ctx->device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(ctx, S2W_ERR_CUDA, "waveforms_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_addr[ctx->device] = p;
  }
  *out = g_noalloc_addr[ctx->device];
  return S2W_OK;
}

}  // namespace

extern "C" int s2w_waveforms_noalloc(s2w_ctx* ctx, const float* slip, float* q, void* stream) {
  if (ctx && ctx->single_pass)
    return fail(ctx, S2W_ERR_UNSUPPORTED, "waveforms_noalloc: not available in the single-pass variant");
  if (!ctx) return S2W_ERR_ARG;
  if (!slip || !q) return fail(ctx, S2W_ERR_ARG, "waveforms_noalloc: slip and q must not be NULL");
  const long long Ns = ctx->Ns, Ng = ctx->Ng, No = ctx->No, Nt = ctx->Nt, Nb = ctx->Nb, Ns_pad = ctx->Ns_pad;
  // the FFT half-length of the context (the single-pass variant, whose L is
  // not 2 Nt, is rejected above)
  const int Lh = static_cast<int>(ctx->L / 2);
  const long long seg_cols = static_cast<long long>(ctx->nseg) * ctx->RL;
  // scratch regions (each 256-byte aligned); FP32_HILO adds a low-order
  // region after each of them
  const int parts = ctx->df ? 2 : 1;
  const size_t sz_s = sizeof(float2) * Nb * Ns_pad, sz_m = sizeof(float2) * Nb * Ng;
  const size_t sz_v = sizeof(float2) * Nb * seg_cols, sz_p = sizeof(float2) * Nb * ctx->nseg * No;
  size_t off[4][2], need = 0;
  const size_t sizes[4] = {sz_s, sz_m, sz_v, sz_p};
  for (int r = 0; r < 4; ++r)
    for (int h = 0; h < 2; ++h) {
      off[r][h] = need;
      if (h < parts) need = align256(need + sizes[r]);
    }
  if (need > kNoAllocScratchBytes)
    return fail(ctx, S2W_ERR_UNSUPPORTED,
                "waveforms_noalloc: this problem needs %zu bytes of scratch, more than the static %zu bytes "
                "(Ns=%lld, Ng=%lld, No=%lld, Nt=%lld); use s2w_waveforms",
                need, kNoAllocScratchBytes, Ns, Ng, No, Nt);
  if (ctx->g_count != ctx->Ng || ctx->p_count != ctx->Ng)
    return fail(ctx, S2W_ERR_STATE, "waveforms_noalloc: operators not fully loaded");
  DeviceGuard guard(ctx->device);
  if (pointer_kind(slip, ctx->device) != 1 || pointer_kind(q, ctx->device) != 1)
    return fail(ctx, S2W_ERR_ARG, "waveforms_noalloc: slip and q must be device pointers of the context's device");
  void* base = nullptr;
  const int rs = noalloc_scratch(ctx, &base);
  if (rs != S2W_OK) return rs;
  unsigned char* sc = static_cast<unsigned char*>(base);
  auto region = [&](int r, int h) { return reinterpret_cast<float2*>(sc + off[r][h]); };
  float2* shat = region(0, 0);
  float2* mhat = region(1, 0);
  float2* vhat = region(2, 0);
  float2* part = region(3, 0);
  float2* shat_lo = ctx->df ? region(0, 1) : nullptr;
  float2* mhat_lo = ctx->df ? region(1, 1) : nullptr;
  float2* vhat_lo = ctx->df ? region(2, 1) : nullptr;
  float2* part_lo = ctx->df ? region(3, 1) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: zero the regions whose
  // padding entries are read (slip spectra columns >= Ns, velocity spectra
  // columns >= Ng); mhat and the partials are overwritten in full.
  CK(cudaMemsetAsync(shat, 0, sz_s, st));
  CK(cudaMemsetAsync(vhat, 0, sz_v, st));
  if (ctx->df) {
    CK(cudaMemsetAsync(shat_lo, 0, sz_s, st));
    CK(cudaMemsetAsync(vhat_lo, 0, sz_v, st));
    CK(launch_df_rfft_rows(slip, Ns, static_cast<int>(Nt), Lh, ctx->tw_df, shat, shat_lo, Ns_pad, Ns, Ns_pad, st));
  } else {
    CK(launch_rfft_rows(slip, Ns, static_cast<int>(Nt), Lh, ctx->tw, shat, Ns_pad, Ns, Ns_pad, st));
  }
  StreamArgs a1{};
  a1.rows = ctx->G;
  a1.rows_lo = ctx->G_lo;
  a1.F = Nb * Ng;
  a1.row_len = static_cast<int>(Ns_pad);
  a1.el = ctx->opts.prec_g;
  a1.x = shat;
  a1.x_lo = shat_lo;
  a1.x_stride = Ns_pad;
  a1.rows_per_vec = Ng;
  a1.scale = ctx->G_scale;
  a1.nblk = ctx->nblk;
  a1.y = mhat;
  a1.y_lo = mhat_lo;
  a1.status = ctx->d_status;
  CK(launch_stream_dot(a1, ctx->num_sms, st));
  if (ctx->df)
    CK(launch_df_retransform(mhat, mhat_lo, Ng, Ng, Lh, ctx->tw_df, 1.0 / ctx->opts.dt, ctx->opts.dt_mode, vhat,
                             vhat_lo, seg_cols, nullptr, st));
  else
    CK(launch_retransform(mhat, Ng, Ng, Lh, ctx->tw, static_cast<float>(1.0 / ctx->opts.dt), ctx->opts.dt_mode, vhat,
                          seg_cols, nullptr, st));
  StreamArgs a2{};
  a2.rows = ctx->P;
  a2.rows_lo = ctx->P_lo;
  a2.F = Nb * ctx->nseg * No;
  a2.row_len = ctx->RL;
  a2.el = ctx->opts.prec_p;
  a2.x = vhat;
  a2.x_lo = vhat_lo;
  a2.x_stride = ctx->RL;
  a2.rows_per_vec = No;
  a2.y = part;
  a2.y_lo = part_lo;
  a2.status = ctx->d_status;
  CK(launch_stream_dot(a2, ctx->num_sms, st));
  if (ctx->df)
    CK(launch_df_reduce_irfft(part, part_lo, 1, static_cast<int>(No), ctx->nseg, Lh, Nb * ctx->nseg * No,
                              static_cast<long long>(ctx->nseg) * No, No, ctx->tw_df, q, st, static_cast<int>(Nt)));
  else
    CK(launch_reduce_irfft(part, 1, static_cast<int>(No), ctx->nseg, Lh, Nb * ctx->nseg * No,
                           static_cast<long long>(ctx->nseg) * No, No, ctx->tw, q, st, static_cast<int>(Nt)));
  ctx->launches += 5;
  return S2W_OK;
}
