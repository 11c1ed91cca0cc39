// Final products of the slide-wise aggregation (Sec. 2.3): the merged label
// map of every tissue class is stained onto the 40x slide in its own colour,
// and the 10x product is resized directly from that stained 40x image.
//
// One pass over the slide: each thread owns an R x R block of 40x pixels
// (R = the resize factor), reads the slide and the class labels covering the
// block once, writes the stained block (optional) and the block's rounded
// mean (optional).  HBM-bound: 3 bytes read + 3 bytes written per 40x pixel,
// plus each class map once.
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

template <int R>
__global__ void __launch_bounds__(128) k_stain(StainArgs a) {
  const int bx = blockIdx.x * 128 + threadIdx.x, by = blockIdx.y;
  const int x0 = bx * R, y0 = by * R;
  if (x0 >= a.W) return;
  const int vx = min(R, a.W - x0), vy = min(R, a.H - y0);
  const bool vec = a.vec != 0;
  int sum[3] = {0, 0, 0};
  for (int dy = 0; dy < vy; ++dy) {
    const int y = y0 + dy;
    uint8_t px[3 * R];
    load_row<R>(a.rgb + (long long)y * a.rs + (long long)x0 * 3, vx, vec, px);
    for (int k = 0; k < a.n; ++k) {
      const uint8_t* lab = a.lab[k];
      if (!lab) continue;
      const int s = a.sh[k];
      const uint8_t* row = lab + (long long)(y >> s) * a.lw[k];
      const int al = a.alpha[k], c0 = a.col[k][0] * al, c1 = a.col[k][1] * al, c2 = a.col[k][2] * al;
      const int inv = 256 - al;
      if ((1 << s) >= R) {
        // the whole row segment lies in one label pixel (R divides f, x0 % R == 0)
        if (__ldg(row + (x0 >> s))) {
#pragma unroll
          for (int i = 0; i < R; ++i) {
            px[3 * i] = (uint8_t)((px[3 * i] * inv + c0 + 128) >> 8);
            px[3 * i + 1] = (uint8_t)((px[3 * i + 1] * inv + c1 + 128) >> 8);
            px[3 * i + 2] = (uint8_t)((px[3 * i + 2] * inv + c2 + 128) >> 8);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i < vx && __ldg(row + ((x0 + i) >> s))) {
            px[3 * i] = (uint8_t)((px[3 * i] * inv + c0 + 128) >> 8);
            px[3 * i + 1] = (uint8_t)((px[3 * i + 1] * inv + c1 + 128) >> 8);
            px[3 * i + 2] = (uint8_t)((px[3 * i + 2] * inv + c2 + 128) >> 8);
          }
        }
      }
    }
    if (a.out) store_row<R>(a.out + (long long)y * a.os + (long long)x0 * 3, vx, vec, px);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (i < vx) {
        sum[0] += px[3 * i];
        sum[1] += px[3 * i + 1];
        sum[2] += px[3 * i + 2];
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
