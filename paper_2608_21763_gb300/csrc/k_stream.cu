// Per-bin complex contractions on the HBM-streaming path (Alg. 2 step 3,
// yhat_l = Fhat_l xhat_l, for a small rupture batch).
//
// Both stages are one kernel.  The resident spectrum is a sequence of F
// contiguous rows of `row_len` complex entries; row f is dotted with the
// vector x_vec(f) = x + (f / rows_per_vec) * x_stride:
//   stage 1: rows (l, i) of Ghat [l][i][Ns_pad], x_vec = shat_l     -> mhat[l][i]
//   stage 2: rows (l, seg, o) of Phat [l][seg][o][RL],
//            x_vec = vhat_l[seg * RL ..]                           -> partial[l][seg][o]
//
// Each CTA owns one contiguous range of rows (balanced to the row) and streams
// it through a 3-stage shared-memory ring filled by cp.async.bulk (one bulk
// copy per stage, L2 evict-first: every operator byte is read exactly once).
// Eight consumer warps take rows in passes: a long row gets a whole warp (lane
// l handles the 16-byte chunks l, l + 32, ..., so a warp reads 512 contiguous
// bytes per step); a short row (a few subfaults) gets a power-of-two group of
// lanes with about four chunks each, several rows per warp pass.  Each lane
// keeps its slice of x_vec in registers across rows that share it.  Products
// accumulate in FP32; FP8 rows are widened exactly to FP16 pairs (one
// conversion per complex entry) and multiplied by the vector held as FP16
// pairs scaled by a power of two (its largest magnitude into [2, 4)), with
// packed FP16 multiply-adds (independent accumulators per lane, each summing
// at most 8 products) flushed into FP32 at the end of the row, so that a
// streamed byte costs about two instructions; long FP8 rows go four per warp
// pass with one butterfly reduction over the lanes for the four;
// the per-(bin, 256-row block) scale and the power of two are undone after
// the dot product.  FP32_HILO rows (hi and lo FP32 arrays) meet
// a vector of pairs (x, x_lo): each product is formed exactly (TwoProduct)
// and summed by TwoSum into double-float accumulators (df.cuh), written as
// pairs (y, y_lo).
#include <type_traits>

#include "df.cuh"
#include "s2w_internal.cuh"

namespace s2w {

namespace {

constexpr int kConsumerWarps = 8;  // the transposed kernel; k_stream_dot takes stream_warps(EL)
constexpr int kStages = 3;
constexpr int kThreads = 32 * (kConsumerWarps + 1);
constexpr int kMaxRowLen = 1024;
constexpr int kStagesT = 2;  // ring depth of the transposed kernel (its reduction buffer needs the room)

template <int EL>
struct Chunk;  // complex entries per 16-byte chunk and how to unpack them

template <>
struct Chunk<EL_FP32> {
  static constexpr int C = 2;
  __device__ __forceinline__ static void unpack(const uint4& u, float2 (&g)[C]) {
    g[0] = make_float2(__uint_as_float(u.x), __uint_as_float(u.y));
    g[1] = make_float2(__uint_as_float(u.z), __uint_as_float(u.w));
  }
};

__device__ __forceinline__ float2 bf2_to_f2(unsigned w) {
  // bf16 -> f32 is exact: the 16 bits move to the top of the word
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <>
struct Chunk<EL_BF16> {
  static constexpr int C = 4;
  __device__ __forceinline__ static void unpack(const uint4& u, float2 (&g)[C]) {
    g[0] = bf2_to_f2(u.x);
    g[1] = bf2_to_f2(u.y);
    g[2] = bf2_to_f2(u.z);
    g[3] = bf2_to_f2(u.w);
  }
};

// Two e4m3 values (bytes 0, 1 of a 16-bit word) widened exactly to an FP16
// pair, and a 32-bit word's two such pairs.
__device__ __forceinline__ __half2 e4m3x2_to_h2(unsigned short v) {
  unsigned r;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(r) : "h"(v));
  return *reinterpret_cast<const __half2*>(&r);
}
__device__ __forceinline__ void e4m3x4_to_h2(unsigned w, __half2& lo, __half2& hi) {
  unsigned short l16, h16;
  asm("mov.b32 {%0, %1}, %2;" : "=h"(l16), "=h"(h16) : "r"(w));
  lo = e4m3x2_to_h2(l16);
  hi = e4m3x2_to_h2(h16);
}

__device__ __forceinline__ float2 fp8x2_to_f2(unsigned short s) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(s), __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

template <>
struct Chunk<EL_FP8> {
  static constexpr int C = 8;
  __device__ __forceinline__ static void unpack(const uint4& u, float2 (&g)[C]) {
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g[2 * k] = fp8x2_to_f2(static_cast<unsigned short>(w[k] & 0xffffu));
      g[2 * k + 1] = fp8x2_to_f2(static_cast<unsigned short>(w[k] >> 16));
    }
  }
};

// EL selects the unpacker (EL_BF16 also serves the hi/lo pair when HILO);
// SHORT: rows of at most 64 chunks, shared by lane groups; DF (with EL_FP32
// and HILO): FP32 pair rows and vectors, double-float sums.
// Consumer warps of k_stream_dot.  FP8 rows carry half the bytes of BF16
// ones, so per-row work (the lane reduction, the scale) weighs more: long FP8
// rows are taken four per warp pass (one reduction for the four), short ones
// by twelve warps (more rows in flight; ~120 registers each, no spills).
__host__ __device__ constexpr int stream_warps(int el, bool short_rows) {
  return (el == EL_FP8 && short_rows) ? 12 : 8;
}

template <int EL, bool HILO, bool SHORT, bool DF = false>
__global__ void __launch_bounds__(32 * (stream_warps(EL, SHORT) + 1), 1)
    k_stream_dot(const StreamArgs a, int stage_rows) {
  constexpr int kConsumerWarps = stream_warps(EL, SHORT);
  static_assert(!DF || (EL == EL_FP32 && HILO), "pair rows: FP32 hi and lo arrays");
  using CH = Chunk<EL>;
  constexpr int C = CH::C;
  // chunk slots per lane: a short row gives each lane at most four chunks
  constexpr int T = SHORT ? 4 : kMaxRowLen / (32 * C);
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);
  uint64_t* empty = full + kStages;
  unsigned char* buf = sm + 128;
  const int row_bytes = a.row_len * (16 / C);
  const int stage_bytes = stage_rows * row_bytes;
  unsigned char* buf_lo = buf + kStages * stage_bytes;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long r0 = a.F * blockIdx.x / gridDim.x;
  const long long r1 = a.F * (blockIdx.x + 1) / gridDim.x;
  const int nst = static_cast<int>((r1 - r0 + stage_rows - 1) / stage_rows);
  const unsigned long long wlim = a.wait_ns ? a.wait_ns : kWaitLimitNs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kConsumerWarps) {  // producer warp: one elected lane issues the copies
    if (lane == 0) {
      const uint64_t pol = l2_policy_evict_first();
      int k = 0;
      for (; k < nst; ++k) {
        const int s = k % kStages;
        if (k >= kStages &&
            !mbar_wait_bounded(empty + s, ((k / kStages) - 1) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY, wlim))
          break;
        if (a.fault_skip && k == 0) continue;  // test hook: stage 0 never fills (no copy, no expected bytes)
        const long long rs = r0 + static_cast<long long>(k) * stage_rows;
        const int nr = static_cast<int>(min(static_cast<long long>(stage_rows), r1 - rs));
        const uint32_t bytes = static_cast<uint32_t>(nr) * row_bytes;
        mbar_arrive_expect_tx(full + s, HILO ? 2 * bytes : bytes);
        bulk_g2s(buf + s * stage_bytes, static_cast<const unsigned char*>(a.rows) + rs * row_bytes, bytes, full + s,
                 pol);
        if (HILO)
          bulk_g2s(buf_lo + s * stage_bytes, static_cast<const unsigned char*>(a.rows_lo) + rs * row_bytes, bytes,
                   full + s, pol);
      }
      // Never leave the CTA with copies in flight: wait for the last stages issued.
      for (int kk = (k > kStages ? k - kStages : 0); kk < k; ++kk)
        mbar_wait_bounded(full + kk % kStages, (kk / kStages) & 1, a.status, DEV_ERR_TIMEOUT_FULL, wlim);
    }
    return;
  }

  // consumer warps: a row is shared by `lpr` lanes (a power of two, chosen so
  // a lane takes about four chunks of a short row), so a warp takes 32 / lpr
  // rows per pass and the row sums need log2(lpr) shuffle steps
  const int nchunk = row_bytes / 16;
  int lpr = 32;
  if (SHORT)
    while (lpr > 1 && 4 * (lpr / 2) >= nchunk) lpr >>= 1;
  const int rpp = 32 / lpr;     // rows per warp pass
  const int sub = lane % lpr;   // lane within its row group
  const int grp = lane / lpr;   // row group within the warp
  constexpr bool F8 = EL == EL_FP8;
  float2 xr[F8 ? 1 : T][F8 ? 1 : C];
  float2 xl[DF ? T : 1][DF ? C : 1];  // DF: low-order parts of x_vec
  // FP8: x_vec times a power of two sx (max |component| into [2, 4)) as FP16
  // pairs (Re, Re) and (Im, Im) for the packed products, and 1 / sx
  __half2 xrr[F8 ? T : 1][F8 ? C : 1], xii[F8 ? T : 1][F8 ? C : 1];
  float x_unscale = 1.f;
  long long vec = -1, vec_end = 0;  // x_vec of rows [vec_end - rows_per_vec, vec_end); rows rise per lane
  if constexpr (F8 && !SHORT) {
    // Long FP8 rows, four per warp pass, all 32 lanes on each: the lane's
    // products of the four rows accumulate side by side (sixteen FP16 pair
    // chains per kind), then one butterfly reduce-scatter over the lanes sums
    // the 8 values (Re and Im of four rows) with 9 shuffles instead of 40;
    // lanes 4v hold value v.  Rows of a pass that fall into the next bin are
    // taken in a second round after the vector reload.
    for (int k = 0; k < nst; ++k) {
      const int s = k % kStages;
      if (!mbar_wait_bounded(full + s, (k / kStages) & 1, a.status, DEV_ERR_TIMEOUT_FULL, wlim)) return;
      const long long rs = r0 + static_cast<long long>(k) * stage_rows;
      const int nr = static_cast<int>(min(static_cast<long long>(stage_rows), r1 - rs));
      for (int base = warp * 4; base < nr; base += kConsumerWarps * 4) {
        int j = 0;
        while (j < 4 && base + j < nr) {
          if (rs + base + j >= vec_end) {  // warp-uniform: every lane works on the same rows
            vec = (rs + base + j) / a.rows_per_vec;
            vec_end = (vec + 1) * a.rows_per_vec;
            const float4* xv = reinterpret_cast<const float4*>(a.x + vec * a.x_stride);
            float amax = 0.f;
#pragma unroll
            for (int t = 0; t < T; ++t) {
              const int c = lane + 32 * t;
#pragma unroll
              for (int q = 0; q < C / 2; ++q) {
                const float4 v = (c < nchunk) ? __ldg(xv + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
              }
            }
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            int e = 0;
            frexpf(amax, &e);  // amax = m 2^e, m in [0.5, 1)
            const float sx = amax > 0.f ? ldexpf(1.f, 2 - e) : 1.f;
            x_unscale = amax > 0.f ? ldexpf(1.f, e - 2) : 1.f;
#pragma unroll
            for (int t = 0; t < T; ++t) {
              const int c = lane + 32 * t;
#pragma unroll
              for (int q = 0; q < C / 2; ++q) {
                const float4 v = (c < nchunk) ? __ldg(xv + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                xrr[t][2 * q] = __float2half2_rn(v.x * sx);
                xii[t][2 * q] = __float2half2_rn(v.y * sx);
                xrr[t][2 * q + 1] = __float2half2_rn(v.z * sx);
                xii[t][2 * q + 1] = __float2half2_rn(v.w * sx);
              }
            }
          }
          int je = j + 1;  // rows j .. je-1 of the pass share this bin's vector
          while (je < 4 && base + je < nr && rs + base + je < vec_end) ++je;
          __half2 ha[4][4], hb[4][4];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) ha[r][q] = hb[r][q] = __float2half2_rn(0.f);
          // ALL: the four rows share the bin (the usual case): no per-row tests
          auto accumulate = [&](auto all_tag) {
            constexpr bool ALL = decltype(all_tag)::value;
#pragma unroll
            for (int t = 0; t < T; ++t) {
              const int c = lane + 32 * t;
              if (c < nchunk) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  if (ALL || (r >= j && r < je)) {
                    const uint4 u =
                        reinterpret_cast<const uint4*>(buf + s * stage_bytes + (base + r) * row_bytes)[c];
                    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                      __half2 g[2];
                      e4m3x4_to_h2(w[q], g[0], g[1]);
#pragma unroll
                      for (int h = 0; h < 2; ++h) {
                        ha[r][q] = __hfma2(g[h], xrr[t][2 * q + h], ha[r][q]);  // (gr xr, gi xr)
                        hb[r][q] = __hfma2(g[h], xii[t][2 * q + h], hb[r][q]);  // (gr xi, gi xi)
                      }
                    }
                  }
                }
              }
            }
          };
          if (j == 0 && je == 4)
            accumulate(std::true_type{});
          else
            accumulate(std::false_type{});
          float v[8];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float2 fa = __half22float2(ha[r][q]), fb = __half22float2(hb[r][q]);
              ar += fa.x - fb.y;
              ai += fb.x + fa.y;
            }
            v[2 * r] = ar;
            v[2 * r + 1] = ai;
          }
          // reduce-scatter: after the step with lane bit b, the lane keeps the
          // half of its values selected by that bit, summed with its partner's
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool up = lane & 16;
            const float keep = up ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, up ? v[i] : v[i + 4], 16);
          }
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const bool up = lane & 8;
            const float keep = up ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, up ? v[i] : v[i + 2], 8);
          }
          {
            const bool up = lane & 4;
            const float keep = up ? v[1] : v[0];
            v[0] = keep + __shfl_xor_sync(0xffffffffu, up ? v[0] : v[1], 4);
          }
          v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
          v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
          const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
          const int r = idx >> 1;
          if ((lane & 3) == 0 && r >= j && r < je) {
            const long long f = rs + base + r;
            const float sc = a.scale[vec * a.nblk + (f - (vec_end - a.rows_per_vec)) / 256] * x_unscale;
            reinterpret_cast<float*>(a.y + f)[idx & 1] = v[0] * sc;
          }
          j = je;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + s);
    }
    return;
  }
  for (int k = 0; k < nst; ++k) {
    const int s = k % kStages;
    if (!mbar_wait_bounded(full + s, (k / kStages) & 1, a.status, DEV_ERR_TIMEOUT_FULL, wlim)) return;
    const long long rs = r0 + static_cast<long long>(k) * stage_rows;
    const int nr = static_cast<int>(min(static_cast<long long>(stage_rows), r1 - rs));
    for (int base = warp * rpp; base < nr; base += kConsumerWarps * rpp) {
      const int lr = base + grp;
      const bool valid = lr < nr;
      const long long f = rs + (valid ? lr : base);
      if (f >= vec_end) {
        vec = f / a.rows_per_vec;
        vec_end = (vec + 1) * a.rows_per_vec;
        const float4* xv = reinterpret_cast<const float4*>(a.x + vec * a.x_stride);
        if constexpr (F8) {
          // two passes over the lane's slice (cached loads): the largest
          // magnitude over the row group's whole vector, then the scaled
          // FP16 pairs; the lanes of one row group take this branch together
          float amax = 0.f;
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const int c = sub + lpr * t;
#pragma unroll
            for (int q = 0; q < C / 2; ++q) {
              const float4 v = (c < nchunk) ? __ldg(xv + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
              amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
          }
          const unsigned gmask = lpr == 32 ? 0xffffffffu : ((1u << lpr) - 1u) << (grp * lpr);  // this row group
          for (int o = lpr / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(gmask, amax, o));
          int e = 0;
          frexpf(amax, &e);  // amax = m 2^e, m in [0.5, 1)
          const float sx = amax > 0.f ? ldexpf(1.f, 2 - e) : 1.f;
          x_unscale = amax > 0.f ? ldexpf(1.f, e - 2) : 1.f;
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const int c = sub + lpr * t;
#pragma unroll
            for (int q = 0; q < C / 2; ++q) {
              const float4 v = (c < nchunk) ? __ldg(xv + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
              xrr[t][2 * q] = __float2half2_rn(v.x * sx);
              xii[t][2 * q] = __float2half2_rn(v.y * sx);
              xrr[t][2 * q + 1] = __float2half2_rn(v.z * sx);
              xii[t][2 * q + 1] = __float2half2_rn(v.w * sx);
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const int c = sub + lpr * t;
#pragma unroll
            for (int q = 0; q < C / 2; ++q) {
              const float4 v = (c < nchunk) ? __ldg(xv + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
              xr[t][2 * q] = make_float2(v.x, v.y);
              xr[t][2 * q + 1] = make_float2(v.z, v.w);
              if constexpr (DF) {
                const float4* xvl = reinterpret_cast<const float4*>(a.x_lo + vec * a.x_stride);
                const float4 w = (c < nchunk) ? __ldg(xvl + c * (C / 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                xl[t][2 * q] = make_float2(w.x, w.y);
                xl[t][2 * q + 1] = make_float2(w.z, w.w);
              }
            }
          }
        }
      }
      const int rrow = valid ? lr : base;
      const uint4* row = reinterpret_cast<const uint4*>(buf + s * stage_bytes + rrow * row_bytes);
      const uint4* row_lo = reinterpret_cast<const uint4*>(buf_lo + s * stage_bytes + rrow * row_bytes);
      if constexpr (DF) {
        // (g + g_lo)(x + x_lo) per complex entry, four real pair products
        // into two compensated accumulators per chain (two chains)
        dacc sr[2] = {{0.f, 0.f}, {0.f, 0.f}}, si[2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int c = sub + lpr * t;
          if (valid && c < nchunk) {
            float2 g[C], gl[C];
            CH::unpack(row[c], g);
            CH::unpack(row_lo[c], gl);
#pragma unroll
            for (int q = 0; q < C; ++q) {
              const dfl gr{g[q].x, gl[q].x}, gi{g[q].y, gl[q].y};
              const dfl xre{xr[t][q].x, xl[t][q].x}, xim{xr[t][q].y, xl[t][q].y};
              acc_mac(sr[q & 1], gr, xre);
              acc_mac(sr[q & 1], df_neg(gi), xim);
              acc_mac(si[q & 1], gr, xim);
              acc_mac(si[q & 1], gi, xre);
            }
          }
        }
        dacc ar = acc_merge(sr[0], sr[1]), ai = acc_merge(si[0], si[1]);
        for (int o = lpr / 2; o > 0; o >>= 1) {
          const dacc br{__shfl_xor_sync(0xffffffffu, ar.s, o), __shfl_xor_sync(0xffffffffu, ar.c, o)};
          const dacc bi{__shfl_xor_sync(0xffffffffu, ai.s, o), __shfl_xor_sync(0xffffffffu, ai.c, o)};
          ar = acc_merge(ar, br);
          ai = acc_merge(ai, bi);
        }
        if (valid && sub == 0) {
          const dfl yr = acc_get(ar), yi = acc_get(ai);
          a.y[f] = make_float2(yr.hi, yi.hi);
          a.y_lo[f] = make_float2(yr.lo, yi.lo);
        }
      } else if constexpr (F8) {
        // e4m3 pairs (Re, Im) widen exactly to FP16 pairs (one cvt per
        // complex entry); g * (xr, xr) and g * (xi, xi) accumulate as FP16
        // pairs over the lane's T = 4 chunks of the row (eight independent
        // accumulator chains of 8 products each: |g| <= 448, |x sx| < 4, so
        // |sum| < 2^14, inside the FP16 range), then into FP32
        static_assert(!F8 || T <= 4, "FP16 accumulation bound: at most 8 products per accumulator");
        float ar = 0.f, ai = 0.f;
        __half2 ha[4], hb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ha[k] = hb[k] = __float2half2_rn(0.f);
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int c = sub + lpr * t;
          if (valid && c < nchunk) {
            const uint4 u = row[c];
            const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              __half2 g[2];
              e4m3x4_to_h2(w[k], g[0], g[1]);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                ha[k] = __hfma2(g[h], xrr[t][2 * k + h], ha[k]);  // (gr xr, gi xr)
                hb[k] = __hfma2(g[h], xii[t][2 * k + h], hb[k]);  // (gr xi, gi xi)
              }
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 fa = __half22float2(ha[k]), fb = __half22float2(hb[k]);
          ar += fa.x - fb.y;
          ai += fb.x + fa.y;
        }
        for (int o = lpr / 2; o > 0; o >>= 1) {
          ar += __shfl_xor_sync(0xffffffffu, ar, o);
          ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (valid && sub == 0) {
          const float sc = a.scale[vec * a.nblk + (f - (vec_end - a.rows_per_vec)) / 256] * x_unscale;
          a.y[f] = make_float2(ar * sc, ai * sc);
        }
      } else {
      float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int c = sub + lpr * t;
        if (valid && c < nchunk) {
          float2 g[C];
          CH::unpack(row[c], g);
          if (HILO) {
            float2 gl[C];
            CH::unpack(row_lo[c], gl);
#pragma unroll
            for (int q = 0; q < C; ++q) g[q] = cadd(g[q], gl[q]);
          }
#pragma unroll
          for (int q = 0; q < C; q += 2) {
            ar0 = fmaf(g[q].x, xr[t][q].x, ar0);
            ar0 = fmaf(-g[q].y, xr[t][q].y, ar0);
            ai0 = fmaf(g[q].x, xr[t][q].y, ai0);
            ai0 = fmaf(g[q].y, xr[t][q].x, ai0);
            ar1 = fmaf(g[q + 1].x, xr[t][q + 1].x, ar1);
            ar1 = fmaf(-g[q + 1].y, xr[t][q + 1].y, ar1);
            ai1 = fmaf(g[q + 1].x, xr[t][q + 1].y, ai1);
            ai1 = fmaf(g[q + 1].y, xr[t][q + 1].x, ai1);
          }
        }
      }
      float ar = ar0 + ar1, ai = ai0 + ai1;
      for (int o = lpr / 2; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
      }
      if (valid && sub == 0) a.y[f] = make_float2(ar, ai);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
}

// Transposed contraction (the adjoint, a correlation with the conjugate
// spectra):  y[u][c] = sum_{f in unit u} conj(rows[f][c]) * w_f.
// A unit is `Rc` consecutive rows of one group of G1 rows (chunk u % nchunk
// of group u / nchunk); the row weight is w[w_base + (g / wa) * wb + (f - g G1)]
// with g = f / G1, times the FP8 row scale when the rows are FP8.
// One CTA per unit at a time; the 8 consumer warps accumulate their rows
// column-wise in registers, then sum across warps through shared memory.
template <int EL, bool HILO>
__global__ void __launch_bounds__(kThreads, 1) k_stream_tdot(const StreamTArgs a, int stage_rows) {
  using CH = Chunk<EL>;
  constexpr int C = CH::C;
  constexpr int T = kMaxRowLen / (32 * C);
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);
  uint64_t* empty = full + kStagesT;
  unsigned char* buf = sm + 128;
  const int row_bytes = a.row_len * (16 / C);
  const int stage_bytes = stage_rows * row_bytes;
  unsigned char* buf_lo = buf + kStagesT * stage_bytes;
  float2* red = reinterpret_cast<float2*>(buf + (HILO ? 2 : 1) * kStagesT * stage_bytes);  // [8][row_len]
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesT; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  auto unit_rows = [&](long long u, long long& f0, long long& f1) {
    const long long g = u / a.nchunk;
    const long long c = u % a.nchunk;
    f0 = g * a.G1 + c * a.Rc;
    f1 = g * a.G1 + min(static_cast<long long>(c + 1) * a.Rc, a.G1);
  };

  if (warp == kConsumerWarps) {
    if (lane == 0) {
      const uint64_t pol = l2_policy_evict_first();
      int it = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
        long long f0, f1;
        unit_rows(u, f0, f1);
        for (long long rs = f0; rs < f1; rs += stage_rows, ++it) {
          const int s = it % kStagesT;
          if (it >= kStagesT &&
              !mbar_wait_bounded(empty + s, ((it / kStagesT) - 1) & 1, a.status, DEV_ERR_TIMEOUT_EMPTY)) {
            ok = false;
            break;
          }
          const int nr = static_cast<int>(min(static_cast<long long>(stage_rows), f1 - rs));
          const uint32_t bytes = static_cast<uint32_t>(nr) * row_bytes;
          mbar_arrive_expect_tx(full + s, HILO ? 2 * bytes : bytes);
          bulk_g2s(buf + s * stage_bytes, static_cast<const unsigned char*>(a.rows) + rs * row_bytes, bytes,
                   full + s, pol);
          if (HILO)
            bulk_g2s(buf_lo + s * stage_bytes, static_cast<const unsigned char*>(a.rows_lo) + rs * row_bytes, bytes,
                     full + s, pol);
        }
      }
      for (int kk = (it > kStagesT ? it - kStagesT : 0); kk < it; ++kk)
        mbar_wait_bounded(full + kk % kStagesT, (kk / kStagesT) & 1, a.status, DEV_ERR_TIMEOUT_FULL);
    }
    return;
  }

  const int nchunk = row_bytes / 16;
  int it = 0;
  for (long long u = blockIdx.x; u < a.n_units; u += gridDim.x) {
    long long f0, f1;
    unit_rows(u, f0, f1);
    float2 acc[T][C];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int q = 0; q < C; ++q) acc[t][q] = make_float2(0.f, 0.f);
    bool ok = true;
    for (long long rs = f0; rs < f1; rs += stage_rows, ++it) {
      const int s = it % kStagesT;
      if (!mbar_wait_bounded(full + s, (it / kStagesT) & 1, a.status, DEV_ERR_TIMEOUT_FULL)) {
        ok = false;
        break;
      }
      const int nr = static_cast<int>(min(static_cast<long long>(stage_rows), f1 - rs));
      for (int lr = warp; lr < nr; lr += kConsumerWarps) {
        const long long f = rs + lr;
        const long long g = f / a.G1;
        const long long within = f - g * a.G1;
        float2 w = a.w[a.w_base + (g / a.wa) * a.wb + within];
        if (EL == EL_FP8) {
          const float sc = a.scale[g * a.nblk + within / 256];
          w.x *= sc;
          w.y *= sc;
        }
        const uint4* row = reinterpret_cast<const uint4*>(buf + s * stage_bytes + lr * row_bytes);
        const uint4* row_lo = reinterpret_cast<const uint4*>(buf_lo + s * stage_bytes + lr * row_bytes);
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int c = lane + 32 * t;
          if (c < nchunk) {
            float2 gv[C];
            CH::unpack(row[c], gv);
            if (HILO) {
              float2 gl[C];
              CH::unpack(row_lo[c], gl);
#pragma unroll
              for (int q = 0; q < C; ++q) gv[q] = cadd(gv[q], gl[q]);
            }
#pragma unroll
            for (int q = 0; q < C; ++q) {  // conj(g) * w
              acc[t][q].x = fmaf(gv[q].x, w.x, fmaf(gv[q].y, w.y, acc[t][q].x));
              acc[t][q].y = fmaf(gv[q].x, w.y, fmaf(-gv[q].y, w.x, acc[t][q].y));
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + s);
    }
    // cross-warp sum of the unit's column accumulators, in fixed warp order
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int c = lane + 32 * t;
      if (c < nchunk)
#pragma unroll
        for (int q = 0; q < C; ++q) red[warp * a.row_len + c * C + q] = acc[t][q];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kConsumerWarps * 32) : "memory");
    for (int col = threadIdx.x; col < a.row_len; col += kConsumerWarps * 32) {
      float2 sum = red[col];
      for (int w2 = 1; w2 < kConsumerWarps; ++w2) sum = cadd(sum, red[w2 * a.row_len + col]);
      a.y[u * a.row_len + col] = sum;
    }
    // second barrier doubles as a vote: if any consumer warp gave up on a
    // wait, all of them leave together (none is left behind on this barrier)
    int any_failed;
    asm volatile(
        "{\n\t.reg .pred pin, pout;\n\t"
        "setp.eq.u32 pin, %1, 0;\n\t"
        "bar.red.or.pred pout, 1, %2, pin;\n\t"
        "selp.u32 %0, 1, 0, pout;\n\t}"
        : "=r"(any_failed)
        : "r"(ok ? 1u : 0u), "r"(kConsumerWarps * 32)
        : "memory");
    if (any_failed) return;
  }
}

template <int EL, bool HILO>
cudaError_t launch_tt(const StreamTArgs& a, int num_sms, cudaStream_t st) {
  constexpr int C = Chunk<EL>::C;
  const int row_bytes = a.row_len * (16 / C);
  const int budget = HILO ? 32 * 1024 : 64 * 1024;
  int stage_rows = budget / row_bytes;
  if (stage_rows >= kConsumerWarps) stage_rows -= stage_rows % kConsumerWarps;
  if (stage_rows < 1) stage_rows = 1;
  const size_t smem = 128 + static_cast<size_t>(kStagesT) * stage_rows * row_bytes * (HILO ? 2 : 1) +
                      sizeof(float2) * kConsumerWarps * a.row_len;
  cudaError_t e = cudaFuncSetAttribute(k_stream_tdot<EL, HILO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  long long grid = num_sms;
  if (grid > a.n_units) grid = a.n_units;
  if (grid < 1) grid = 1;
  k_stream_tdot<EL, HILO><<<static_cast<unsigned>(grid), kThreads, smem, st>>>(a, stage_rows);
  return cudaGetLastError();
}

template <int EL, bool HILO, bool SHORT, bool DF = false>
cudaError_t launch_t(const StreamArgs& a, int num_sms, cudaStream_t st) {
  constexpr int C = Chunk<EL>::C;
  const int row_bytes = a.row_len * (16 / C);
  const int budget = HILO ? 32 * 1024 : 64 * 1024;
  int stage_rows = budget / row_bytes;
  if (stage_rows >= 8) stage_rows -= stage_rows % 8;
  if (stage_rows < 1) stage_rows = 1;
  const size_t smem = 128 + static_cast<size_t>(kStages) * stage_rows * row_bytes * (HILO ? 2 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_stream_dot<EL, HILO, SHORT, DF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  long long grid = num_sms;
  if (grid > a.F) grid = a.F;
  if (grid < 1) grid = 1;
  k_stream_dot<EL, HILO, SHORT, DF><<<static_cast<unsigned>(grid), 32 * (stream_warps(EL, SHORT) + 1), smem, st>>>(
      a, stage_rows);
  return cudaGetLastError();
}

// Rows of at most 64 16-byte chunks (C complex entries each) take the
// lane-group variant.
bool short_rows(const StreamArgs& a, int C) { return a.row_len / C <= 64; }

}  // namespace

cudaError_t launch_stream_dot(const StreamArgs& a, int num_sms, cudaStream_t st) {
  if (a.F <= 0) return cudaSuccess;
  if (a.row_len <= 0 || a.row_len > kMaxRowLen || (a.row_len % 8) != 0) return cudaErrorInvalidValue;
  switch (a.el) {
    case EL_FP32:
      return short_rows(a, 2) ? launch_t<EL_FP32, false, true>(a, num_sms, st)
                              : launch_t<EL_FP32, false, false>(a, num_sms, st);
    case EL_BF16:
      return short_rows(a, 4) ? launch_t<EL_BF16, false, true>(a, num_sms, st)
                              : launch_t<EL_BF16, false, false>(a, num_sms, st);
    case EL_BF16_HILO:
      return short_rows(a, 4) ? launch_t<EL_BF16, true, true>(a, num_sms, st)
                              : launch_t<EL_BF16, true, false>(a, num_sms, st);
    case EL_FP8:
      return short_rows(a, 8) ? launch_t<EL_FP8, false, true>(a, num_sms, st)
                              : launch_t<EL_FP8, false, false>(a, num_sms, st);
    case EL_FP32_HILO:
      if (a.rows_lo == nullptr || a.x_lo == nullptr || a.y_lo == nullptr) return cudaErrorInvalidValue;
      return short_rows(a, 2) ? launch_t<EL_FP32, true, true, true>(a, num_sms, st)
                              : launch_t<EL_FP32, true, false, true>(a, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace s2w

namespace s2w {

cudaError_t launch_stream_tdot(const StreamTArgs& a, int num_sms, cudaStream_t st) {
  if (a.n_units <= 0) return cudaSuccess;
  if (a.row_len <= 0 || a.row_len > kMaxRowLen || (a.row_len % 8) != 0 || a.Rc < 1 || a.nchunk < 1)
    return cudaErrorInvalidValue;
  switch (a.el) {
    case EL_FP32: return launch_tt<EL_FP32, false>(a, num_sms, st);
    case EL_BF16: return launch_tt<EL_BF16, false>(a, num_sms, st);
    case EL_BF16_HILO: return launch_tt<EL_BF16, true>(a, num_sms, st);
    case EL_FP8: return launch_tt<EL_FP8, false>(a, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace s2w
