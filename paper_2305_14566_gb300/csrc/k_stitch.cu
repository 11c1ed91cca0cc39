// Slide-wise aggregation (Sec. 2.3) of the overlapping tile predictions
// (Sec. 2.2, Sec. 3.2): every output pixel is owned by exactly one thread,
// which reads the logits of the processed tiles covering it in ascending
// (row, column) tile order, so no atomics are used and the result is
// deterministic.  The same pass emits the labels:
//   average mode: label = cov > 0 and mean logit > 0
//   vote mode:    label = cov > 0 and 2 * (#tiles with logit > 0) >= cov
// optionally ANDed with the tissue foreground (Sec. 2.3), plus the optional
// stitched logits, coverage and per-scale argmax map.
// Each thread handles four consecutive pixels with 16-byte loads when the
// crop is 4-aligned (tile borders fall on multiples of the stride S, S % 4 == 0).
// With a stitch window the average is weighted: L = sum_p w_p l_p / sum_p w_p,
// w_p = t(y - y_p) t(x - x_p) from a P-entry table (votes stay unweighted).
// A launch covers one band of output rows: the slide is stitched band by band
// as soon as the tile rows covering a band are done, and the tile logits live
// in a ring of slots (foreground index mod slot_cap) that holds only the tile
// rows a band still needs.
#include "omni_internal.cuh"

namespace omni {
namespace {

// Classes are the outer loop so only one class's sums and votes are live
// (the tile slots are re-read per class from L1); this keeps the register
// count low enough for the occupancy a bandwidth-bound pass needs.  FEW: at
// most 2 x 2 tiles cover a pixel (P <= 2 S); their ring slots and offsets are
// then resolved once per thread, not once per class.
template <bool VEC, bool WIN, bool FEW>
__global__ void __launch_bounds__(256) k_stitch(StitchArgs a) {
  constexpr int NV = VEC ? 4 : 1;
  const int ox = (blockIdx.x * 64 + (threadIdx.x & 63)) * NV;
  const int oy = a.row0 + blockIdx.y * 4 + (threadIdx.x >> 6);
  if (oy >= a.row0 + a.nrows || oy >= a.oh || ox >= a.ow) return;
  const int cy = oy + a.oy0, cx = ox + a.ox0;
  const long long PP = (long long)a.P * a.P;
  const int i_lo = max(0, (cy - a.P) / a.S + ((cy - a.P) >= 0 ? 1 : 0));
  const int i_hi = min(a.gh - 1, cy / a.S);
  const int j_lo = max(0, (cx - a.P) / a.S + ((cx - a.P) >= 0 ? 1 : 0));
  const int j_hi = min(a.gw - 1, cx / a.S);

  bool tis = true;
  if (a.tissue) {
    const int ty = (int)(((long long)cy * a.f) / kThumb), tx = (int)(((long long)cx * a.f) / kThumb);
    tis = a.tissue[(long long)ty * a.tw + tx] != 0;
  }
  const long long o = (long long)oy * a.ow + ox;
  float best[NV];
  int arg[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { best[v] = 0.f; arg[v] = 0; }
  int cov = 0;
  long long toff[4] = {0, 0, 0, 0};       // FEW: covering tiles' class-0 logit offsets
  int txo[4] = {0, 0, 0, 0};              // ... their column offset into the window table
  float twy[4] = {1.f, 1.f, 1.f, 1.f};    // ... and their row weight
  int nt = 0;
  if constexpr (FEW) {
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const int i = i_lo + di, j = j_lo + dj;
        if (i > i_hi || j > j_hi) continue;
        int slot = a.slot_map[i * a.gw + j];
        if (slot < 0) continue;
        if (a.slot_cap) slot = (slot + a.slot_base) % a.slot_cap;
        const int k = di * 2 + dj;         // fixed register index; unused entries stay cold
        toff[k] = (long long)slot * a.n_cls * PP + (long long)(cy - i * a.S) * a.P + (cx - j * a.S);
        txo[k] = cx - j * a.S;
        if (WIN) twy[k] = __ldg(a.window + (cy - i * a.S));
        nt |= 1 << k;
      }
  }
  for (int c = 0; c < a.n_cls; ++c) {
    float sum[NV], wsum[NV];
    int votes[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { sum[v] = 0.f; wsum[v] = 0.f; votes[v] = 0; }
    int n = 0;
    if constexpr (FEW) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!(nt >> k & 1)) continue;
        ++n;
        const float* base = a.logits + toff[k] + (long long)c * PP;
        float l[NV];
        if constexpr (VEC) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(base));
          l[0] = q.x; l[1] = q.y; l[2] = q.z; l[3] = q.w;
        } else {
          l[0] = __ldg(base);
        }
        float w[NV];
        if constexpr (WIN && VEC) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(a.window + txo[k]));
          w[0] = twy[k] * q.x; w[1] = twy[k] * q.y; w[2] = twy[k] * q.z; w[3] = twy[k] * q.w;
        } else if constexpr (WIN) {
          w[0] = twy[k] * __ldg(a.window + txo[k]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WIN) {
            sum[v] = fmaf(w[v], l[v], sum[v]);
            wsum[v] += w[v];
          } else {
            sum[v] += l[v];
          }
          votes[v] += l[v] > 0.f ? 1 : 0;
        }
      }
    }
    for (int i = i_lo; i <= i_hi && !FEW; ++i) {
      const float wy = WIN ? __ldg(a.window + (cy - i * a.S)) : 1.f;
      // the covering tiles' loads are independent: unrolled, several are in
      // flight per thread (the pass is bound by memory latency otherwise)
#pragma unroll 4
      for (int j = j_lo; j <= j_hi; ++j) {
        int slot = a.slot_map[i * a.gw + j];
        if (slot < 0) continue;
        if (a.slot_cap) slot = (slot + a.slot_base) % a.slot_cap;
        ++n;
        const float* base = a.logits + ((long long)slot * a.n_cls + c) * PP +
                            (long long)(cy - i * a.S) * a.P + (cx - j * a.S);
        float l[NV];
        if constexpr (VEC) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(base));
          l[0] = q.x; l[1] = q.y; l[2] = q.z; l[3] = q.w;
        } else {
          l[0] = __ldg(base);
        }
        float w[NV];
        if constexpr (WIN && VEC) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(a.window + (cx - j * a.S)));
          w[0] = wy * q.x; w[1] = wy * q.y; w[2] = wy * q.z; w[3] = wy * q.w;
        } else if constexpr (WIN) {
          w[0] = wy * __ldg(a.window + (cx - j * a.S));
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WIN) {
            sum[v] = fmaf(w[v], l[v], sum[v]);
            wsum[v] += w[v];
          } else {
            sum[v] += l[v];
          }
          votes[v] += l[v] > 0.f ? 1 : 0;
        }
      }
    }
    cov = n;
    float L[NV];
    uint8_t lab[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (WIN) L[v] = cov > 0 ? sum[v] / wsum[v] : 0.f;
      else L[v] = cov > 0 ? sum[v] / (float)cov : 0.f;
      const bool on = a.mode == OMNI_STITCH_AVG ? (cov > 0 && L[v] > 0.f) : (cov > 0 && 2 * votes[v] >= cov);
      lab[v] = (on && tis) ? 1 : 0;
      if (L[v] > best[v]) { best[v] = L[v]; arg[v] = a.cls_ids[c] + 1; }
    }
    if (a.labels[c]) {
      if constexpr (VEC) {
        *reinterpret_cast<uchar4*>(a.labels[c] + o) = make_uchar4(lab[0], lab[1], lab[2], lab[3]);
      } else {
        a.labels[c][o] = lab[0];
      }
    }
    if (a.out_logits[c]) {
      if constexpr (VEC) {
        *reinterpret_cast<float4*>(a.out_logits[c] + o) = make_float4(L[0], L[1], L[2], L[3]);
      } else {
        a.out_logits[c][o] = L[0];
      }
    }
  }
  if (a.coverage) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a.coverage[o + v] = (uint16_t)cov;
  }
  if (a.argmax) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a.argmax[o + v] = (uint8_t)arg[v];
  }
}

}  // namespace

cudaError_t launch_stitch(const StitchArgs& a, cudaStream_t st) {
  if (a.n_cls < 1 || a.n_cls > OMNI_MAX_CLASSES) return cudaErrorInvalidValue;
  if (a.oh <= 0 || a.ow <= 0 || a.nrows <= 0) return cudaSuccess;
  if (a.row0 < 0 || a.slot_cap < 0) return cudaErrorInvalidValue;
  const bool vec = (a.ow % 4 == 0) && (a.ox0 % 4 == 0) && (a.S % 4 == 0) && (a.P % 4 == 0);
  const bool few = a.P <= 2 * a.S;
  if (vec) {
    dim3 grid((a.ow / 4 + 63) / 64, (a.nrows + 3) / 4);
    if (few) {
      if (a.window) k_stitch<true, true, true><<<grid, 256, 0, st>>>(a);
      else k_stitch<true, false, true><<<grid, 256, 0, st>>>(a);
    } else {
      if (a.window) k_stitch<true, true, false><<<grid, 256, 0, st>>>(a);
      else k_stitch<true, false, false><<<grid, 256, 0, st>>>(a);
    }
  } else {
    dim3 grid((a.ow + 63) / 64, (a.nrows + 3) / 4);
    if (few) {
      if (a.window) k_stitch<false, true, true><<<grid, 256, 0, st>>>(a);
      else k_stitch<false, false, true><<<grid, 256, 0, st>>>(a);
    } else {
      if (a.window) k_stitch<false, true, false><<<grid, 256, 0, st>>>(a);
      else k_stitch<false, false, false><<<grid, 256, 0, st>>>(a);
    }
  }
  return cudaGetLastError();
}

}  // namespace omni
