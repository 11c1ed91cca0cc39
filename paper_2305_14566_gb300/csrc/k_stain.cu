// Final products of the slide-wise aggregation (Sec. 2.3): the merged label
// map of every tissue class is stained onto the 40x slide in its own colour,
// and the 10x product is resized directly from that stained 40x image.
//
// One pass over the slide: each thread owns an R x R block of 40x pixels
// (R = the resize factor), reads the block's slide pixels, then per class the
// labels covering the block (all loads of a class issued together), writes
// the stained block (optional) and the block's rounded mean (optional).
// HBM-bound: 3 bytes read + 3 bytes written per 40x pixel, plus each class
// map once.
#include "omni_internal.cuh"

namespace omni {
namespace {

struct StainArgs {
  const uint8_t* rgb; long long rs;
  int H, W;
  int n;
  const uint8_t* lab[OMNI_MAX_CLASSES];
  int lw[OMNI_MAX_CLASSES];            // label map row length ceil(W / f)
  int sh[OMNI_MAX_CLASSES];            // log2 f
  int col[OMNI_MAX_CLASSES][3];
  int alpha[OMNI_MAX_CLASSES];         // 0..256
  int lvec[OMNI_MAX_CLASSES];          // 1: label rows may be read as 4-byte words
  uint8_t* out; long long os;          // stained 40x, or null
  uint8_t* down; long long ds;         // R x R rounded mean, or null
  int vec;                             // 1: rows may use 4-byte loads / stores
};

template <int R>
__device__ __forceinline__ void load_row(const uint8_t* p, int valid, bool vec, uint8_t (&px)[3 * R]) {
  if constexpr (R % 4 == 0) {
    if (vec && valid == R) {
#pragma unroll
      for (int q = 0; q < 3 * R / 4; ++q) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p) + q);
        px[4 * q] = w & 255; px[4 * q + 1] = (w >> 8) & 255;
        px[4 * q + 2] = (w >> 16) & 255; px[4 * q + 3] = w >> 24;
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < 3 * R; ++i) px[i] = i < 3 * valid ? __ldg(p + i) : 0;
}

template <int R>
__device__ __forceinline__ void store_row(uint8_t* p, int valid, bool vec, const uint8_t (&px)[3 * R]) {
  if constexpr (R % 4 == 0) {
    if (vec && valid == R) {
#pragma unroll
      for (int q = 0; q < 3 * R / 4; ++q)
        reinterpret_cast<uint32_t*>(p)[q] = (uint32_t)px[4 * q] | ((uint32_t)px[4 * q + 1] << 8) |
                                            ((uint32_t)px[4 * q + 2] << 16) | ((uint32_t)px[4 * q + 3] << 24);
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < 3 * R; ++i)
    if (i < 3 * valid) p[i] = px[i];
}

// Labels of one class over G rows of the thread's R x R block, one bit per
// pixel (bit i of on[dy] = pixel (dy, i) of the group).  Every load of the
// group is issued before any is used, so a class costs one memory latency,
// not one per row.
template <int R, int G>
__device__ __forceinline__ void class_bits(const StainArgs& a, int k, int x0, int y0, int vx, int vy,
                                           uint32_t (&on)[G]) {
  const uint8_t* lab = a.lab[k];
  const int s = a.sh[k];
  const long long lw = a.lw[k];
  if ((1 << s) >= R) {
    // R divides f and the block origin is a multiple of R: one label pixel covers the block
    const uint32_t v = __ldg(lab + (long long)(y0 >> s) * lw + (x0 >> s));
    const uint32_t m = v ? (1u << R) - 1u : 0u;
#pragma unroll
    for (int dy = 0; dy < G; ++dy) on[dy] = m;
    return;
  }
  uint32_t raw[G][R];
  if constexpr (R % 4 == 0) {
    if (s == 0 && a.lvec[k] && vx == R) {
      // a map at the slide's own scale: R consecutive label bytes per row, read as words
#pragma unroll
      for (int dy = 0; dy < G; ++dy) {
#pragma unroll
        for (int w = 0; w < R / 4; ++w) {
          const uint32_t q =
              dy < vy ? __ldg(reinterpret_cast<const uint32_t*>(lab + (long long)(y0 + dy) * lw + x0) + w) : 0u;
          raw[dy][4 * w] = q & 255u;
          raw[dy][4 * w + 1] = (q >> 8) & 255u;
          raw[dy][4 * w + 2] = (q >> 16) & 255u;
          raw[dy][4 * w + 3] = q >> 24;
        }
      }
#pragma unroll
      for (int dy = 0; dy < G; ++dy) {
        uint32_t m = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) m |= (raw[dy][i] ? 1u : 0u) << i;
        on[dy] = m;
      }
      return;
    }
  }
  // f < R: pixel i reads label column (x0 + i) / f (neighbouring pixels may share it)
#pragma unroll
  for (int dy = 0; dy < G; ++dy) {
    const uint8_t* row = lab + (long long)((y0 + dy) >> s) * lw;
#pragma unroll
    for (int i = 0; i < R; ++i) raw[dy][i] = (dy < vy && i < vx) ? (uint32_t)__ldg(row + ((x0 + i) >> s)) : 0u;
  }
#pragma unroll
  for (int dy = 0; dy < G; ++dy) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) m |= (raw[dy][i] ? 1u : 0u) << i;
    on[dy] = m;
  }
}

// The block is processed G rows at a time (G * 3R bytes of pixels stay in
// registers): all of it for R = 2 and 4, two rows at a time for R = 8.
template <int R>
__global__ void __launch_bounds__(128) k_stain(StainArgs a) {
  constexpr int G = R >= 8 ? 2 : R;
  const int bx = blockIdx.x * 128 + threadIdx.x, by = blockIdx.y;
  const int x0 = bx * R, y0 = by * R;
  if (x0 >= a.W) return;
  const int vx = min(R, a.W - x0), vy = min(R, a.H - y0);
  const bool vec = a.vec != 0;
  int sum[3] = {0, 0, 0};
#pragma unroll 1
  for (int g0 = 0; g0 < vy; g0 += G) {
    const int gy = y0 + g0, gv = vy - g0;        // first row and valid rows of the group
    uint8_t px[G][3 * R];
#pragma unroll
    for (int dy = 0; dy < G; ++dy) {
      if (dy < gv) {
        load_row<R>(a.rgb + (long long)(gy + dy) * a.rs + (long long)x0 * 3, vx, vec, px[dy]);
      } else {
#pragma unroll
        for (int i = 0; i < 3 * R; ++i) px[dy][i] = 0;
      }
    }
    for (int k = 0; k < a.n; ++k) {
      if (!a.lab[k]) continue;
      uint32_t on[G];
      class_bits<R, G>(a, k, x0, gy, vx, gv, on);
      const int al = a.alpha[k], inv = 256 - al;
      const int c0 = a.col[k][0] * al + 128, c1 = a.col[k][1] * al + 128, c2 = a.col[k][2] * al + 128;
#pragma unroll
      for (int dy = 0; dy < G; ++dy) {
        if (!on[dy]) continue;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if ((on[dy] >> i) & 1u) {
            px[dy][3 * i] = (uint8_t)((px[dy][3 * i] * inv + c0) >> 8);
            px[dy][3 * i + 1] = (uint8_t)((px[dy][3 * i + 1] * inv + c1) >> 8);
            px[dy][3 * i + 2] = (uint8_t)((px[dy][3 * i + 2] * inv + c2) >> 8);
          }
        }
      }
    }
#pragma unroll
    for (int dy = 0; dy < G; ++dy) {
      if (dy < gv) {
        if (a.out) store_row<R>(a.out + (long long)(gy + dy) * a.os + (long long)x0 * 3, vx, vec, px[dy]);
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i < vx) {
            sum[0] += px[dy][3 * i];
            sum[1] += px[dy][3 * i + 1];
            sum[2] += px[dy][3 * i + 2];
          }
        }
      }
    }
  }
  if (a.down) {
    const int n = vx * vy;
    uint8_t* d = a.down + (long long)by * a.ds + (long long)bx * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = (uint8_t)((sum[c] + n / 2) / n);
  }
}

}  // namespace
}  // namespace omni

using namespace omni;

extern "C" omni_status omni_stain(const uint8_t* rgb_dev, int32_t H, int32_t W, int64_t row_stride,
                                  int32_t n_maps, const uint8_t* const* labels_dev, const int32_t* factors,
                                  const uint8_t* colours, const int32_t* alpha, uint8_t* out40_dev,
                                  int64_t out40_stride, int32_t down, uint8_t* outd_dev, int64_t outd_stride,
                                  void* stream) {
  if (!rgb_dev || H <= 0 || W <= 0 || row_stride < (int64_t)W * 3) return OMNI_EINVAL;
  if (n_maps < 0 || n_maps > OMNI_MAX_CLASSES || (n_maps && (!labels_dev || !factors || !colours || !alpha)))
    return OMNI_EINVAL;
  if (!out40_dev && !outd_dev) return OMNI_EINVAL;
  if (out40_dev && out40_stride < (int64_t)W * 3) return OMNI_EINVAL;
  const int R = outd_dev ? down : 4;
  if (R != 2 && R != 4 && R != 8) return OMNI_EINVAL;
  if (outd_dev && outd_stride < (int64_t)((W + R - 1) / R) * 3) return OMNI_EINVAL;
  StainArgs a{};
  a.rgb = rgb_dev; a.rs = row_stride; a.H = H; a.W = W; a.n = n_maps;
  for (int k = 0; k < n_maps; ++k) {
    const int f = factors[k];
    if (f != 1 && f != 2 && f != 4 && f != 8) return OMNI_EINVAL;
    if (alpha[k] < 0 || alpha[k] > 256) return OMNI_EINVAL;
    a.lab[k] = labels_dev[k];
    a.lw[k] = (W + f - 1) / f;
    a.sh[k] = f == 1 ? 0 : f == 2 ? 1 : f == 4 ? 2 : 3;
    for (int c = 0; c < 3; ++c) a.col[k][c] = colours[3 * k + c];
    a.alpha[k] = alpha[k];
    a.lvec[k] = a.lab[k] && reinterpret_cast<uintptr_t>(a.lab[k]) % 4 == 0 && a.lw[k] % 4 == 0;
  }
  a.out = out40_dev; a.os = out40_stride;
  a.down = outd_dev; a.ds = outd_stride;
  a.vec = (row_stride % 4 == 0) && (reinterpret_cast<uintptr_t>(rgb_dev) % 4 == 0) &&
          (!out40_dev || ((out40_stride % 4 == 0) && (reinterpret_cast<uintptr_t>(out40_dev) % 4 == 0)));
  const int bw = (W + R - 1) / R, bh = (H + R - 1) / R;
  if (bh > 65535) return OMNI_EINVAL;
  dim3 grid((bw + 127) / 128, bh);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (R) {
    case 2: k_stain<2><<<grid, 128, 0, st>>>(a); break;
    case 4: k_stain<4><<<grid, 128, 0, st>>>(a); break;
    default: k_stain<8><<<grid, 128, 0, st>>>(a); break;
  }
  return cudaGetLastError() == cudaSuccess ? OMNI_OK : OMNI_ECUDA;
}
