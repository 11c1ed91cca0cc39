// Omni-Seg dynamic head (Sec. 2.2): a controller turns the tile's global
// average-pooled bottleneck feature plus one-hot class and scale codes into the
// 153 parameters of a per-tile, per-class 1x1 head 8 -> 8 -> 8 -> 1, which is
// applied at every pixel of the pre-head feature h0 = ReLU(Wh y0 + bh).
//
// k_gap_controller reduces the bottleneck of a tile to its channel means and
// evaluates theta for every class of the scale in the same launch (one CTA per
// tile); k_head runs the pre-head and all heads of the scale over the tile
// pixels, writing FP32 logits, where the last decoder conv does not run them
// in its epilogue.
#include <algorithm>

#include <cuda_fp16.h>

#include "omni_internal.cuh"

namespace omni {
namespace {

constexpr int kHeadThreads = 128;
constexpr int kPixPerBlock = 4096;

template <typename T> struct Load8;
template <> struct Load8<float> {
  static __device__ __forceinline__ void f(const float* p, float v[8]) {
    const float4 x = *reinterpret_cast<const float4*>(p), y = *reinterpret_cast<const float4*>(p + 4);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  }
};
template <> struct Load8<__nv_bfloat16> {
  static __device__ __forceinline__ void f(const __nv_bfloat16* p, float v[8]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

template <> struct Load8<__half> {
  static __device__ __forceinline__ void f(const __half* p, float v[8]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

// One CTA per tile.  GAP: thread t owns the channel octet 8 (t mod octets)
// .. +7 and the pixels p = phase (mod phases), read as one 16-byte vector per
// pixel; the phases' partial sums are added in phase order, so the result does
// not depend on scheduling.  Controller: theta[ci][i] = Wc[i] . g + bc[i] +
// Wc[i][Cb + n_classes + s] + Wc[i][Cb + class]; warp w takes rows w, w + 16,
// ..., its lanes stride over the row and a fixed shuffle tree sums them.
constexpr int kGcThreads = 512;
template <typename T>
__global__ void __launch_bounds__(kGcThreads) k_gap_controller(HeadArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int Cb = a.Cb, octets = Cb / 8;
  const int phases = max(1, kGcThreads / octets);
  float* part = sm;                       // [phases][Cb]
  float* g = sm + phases * Cb;            // [Cb]
  const int b = blockIdx.x, t = threadIdx.x;
  const int RR = a.Rb * a.Rb;
  const int oc = t % octets, ph = t / octets;
  if (ph < phases) {
    const T* base = static_cast<const T*>(a.bott) + (long long)b * RR * Cb + 8 * oc;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int p = ph; p < RR; p += phases) {
      float v[8];
      Load8<T>::f(base + (long long)p * Cb, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += v[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) part[ph * Cb + 8 * oc + q] = acc[q];
  }
  __syncthreads();
  for (int c = t; c < Cb; c += kGcThreads) {
    float s = 0.f;
    for (int h = 0; h < phases; ++h) s += part[h * Cb + c];
    g[c] = s / (float)RR;
    if (a.gap_out) a.gap_out[(long long)b * Cb + c] = g[c];
  }
  __syncthreads();
  const int lane = t & 31, warp = t >> 5, nw = kGcThreads / 32;
  const int zdim = Cb + a.n_classes + a.n_scales;
  for (int row = warp; row < kHeadParams; row += nw) {
    const float* w = a.wc + (long long)row * zdim;
    float s = 0.f;
    for (int k = lane; k < Cb; k += 32) s = fmaf(w[k], g[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float common = s + w[Cb + a.n_classes + a.scale] + a.bc[row];
    for (int ci = lane; ci < a.n_cls_here; ci += 32)
      a.theta[((long long)b * a.n_cls_here + ci) * kHeadParams + row] = common + w[Cb + a.cls_ids[ci]];
  }
}

// Each thread evaluates kHeadPx pixels (kHeadThreads apart, so a warp's loads
// cover consecutive pixels) and reuses every weight it reads from shared
// memory for all of them; theta rows are padded to 160 floats so they are
// 16-byte aligned for vector loads.
constexpr int kHeadPx = 4;
constexpr int kThetaStride = 160;

template <int C0, typename T>
__global__ void __launch_bounds__(kHeadThreads) k_head(HeadArgs a) {
  __shared__ __align__(16) float theta[OMNI_MAX_CLASSES][kThetaStride];
  __shared__ __align__(16) float wh[kHeadCh * C0];
  __shared__ float bh[kHeadCh];
  const int b = blockIdx.y;
  const int t = threadIdx.x;
  for (int i = t; i < kHeadCh * C0; i += kHeadThreads) wh[i] = a.wh[i];
  if (t < kHeadCh) bh[t] = a.bh[t];
  for (int i = t; i < a.n_cls_here * kHeadParams; i += kHeadThreads)
    theta[i / kHeadParams][i % kHeadParams] = a.theta[(long long)b * a.n_cls_here * kHeadParams + i];
  __syncthreads();

  const long long PP = (long long)a.P * a.P;
  const T* Y = static_cast<const T*>(a.y0) + (long long)b * PP * C0;
  float* out = a.logits + (long long)(a.slot0 + b) * a.n_cls_here * PP;
  const long long p0 = (long long)blockIdx.x * kPixPerBlock;
  for (int q0 = 0; q0 < kPixPerBlock; q0 += kHeadThreads * kHeadPx) {
    long long pix[kHeadPx];
    bool live[kHeadPx];
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u) {
      pix[u] = p0 + q0 + u * kHeadThreads + t;
      live[u] = pix[u] < PP;
    }
    if (!live[0]) break;
    float h0[kHeadPx][kHeadCh];
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u)
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) h0[u][o] = bh[o];
#pragma unroll
    for (int c0 = 0; c0 < C0; c0 += 8) {
      float y[kHeadPx][8];
#pragma unroll
      for (int u = 0; u < kHeadPx; ++u) {
        if (live[u]) Load8<T>::f(Y + pix[u] * C0 + c0, y[u]);
        else
#pragma unroll
          for (int c = 0; c < 8; ++c) y[u][c] = 0.f;
      }
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&wh[o * C0 + c0]);
        const float4 w1 = *reinterpret_cast<const float4*>(&wh[o * C0 + c0 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int u = 0; u < kHeadPx; ++u) h0[u][o] = fmaf(w[c], y[u][c], h0[u][o]);
      }
    }
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u)
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) h0[u][o] = fmaxf(h0[u][o], 0.f);
    for (int ci = 0; ci < a.n_cls_here; ++ci) {
      const float* th = theta[ci];
      float h1[kHeadPx][kHeadCh], h2[kHeadPx][kHeadCh];
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&th[o * 8]);
        const float4 w1 = *reinterpret_cast<const float4*>(&th[o * 8 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float bias = th[136 + o];
#pragma unroll
        for (int u = 0; u < kHeadPx; ++u) {
          float s = bias;
#pragma unroll
          for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h0[u][c], s);
          h1[u][o] = fmaxf(s, 0.f);
        }
      }
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&th[64 + o * 8]);
        const float4 w1 = *reinterpret_cast<const float4*>(&th[64 + o * 8 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float bias = th[144 + o];
#pragma unroll
        for (int u = 0; u < kHeadPx; ++u) {
          float s = bias;
#pragma unroll
          for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h1[u][c], s);
          h2[u][o] = fmaxf(s, 0.f);
        }
      }
      const float4 w0 = *reinterpret_cast<const float4*>(&th[128]);
      const float4 w1 = *reinterpret_cast<const float4*>(&th[132]);
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int u = 0; u < kHeadPx; ++u) {
        float s = th[152];
#pragma unroll
        for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h2[u][c], s);
        if (live[u]) out[ci * PP + pix[u]] = s;
      }
    }
  }
}

template <typename T>
cudaError_t head_t(const HeadArgs& a, cudaStream_t st) {
  long long PP = (long long)a.P * a.P;
  dim3 grid((unsigned)((PP + kPixPerBlock - 1) / kPixPerBlock), a.B);
  switch (a.C0) {
    case 8: k_head<8, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 16: k_head<16, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 32: k_head<32, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 64: k_head<64, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gap_controller(const HeadArgs& a, cudaStream_t st) {
  if (a.n_cls_here < 1 || a.n_cls_here > OMNI_MAX_CLASSES || a.B < 1 || !a.bott || a.Rb < 1) return cudaErrorInvalidValue;
  if (a.Cb < 8 || a.Cb % 8 || a.Cb / 8 > kGcThreads) return cudaErrorInvalidValue;
  if (reinterpret_cast<uintptr_t>(a.bott) % 16) return cudaErrorInvalidValue;
  const int phases = std::max(1, kGcThreads / (a.Cb / 8));
  const size_t smem = (size_t)(phases + 1) * a.Cb * sizeof(float);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  if (a.precision == OMNI_FP32)
    k_gap_controller<float><<<a.B, kGcThreads, smem, st>>>(a);
  else if (a.precision == OMNI_FP16)
    k_gap_controller<__half><<<a.B, kGcThreads, smem, st>>>(a);
  else
    k_gap_controller<__nv_bfloat16><<<a.B, kGcThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_head(const HeadArgs& a, cudaStream_t st) {
  if (a.n_cls_here < 1 || a.n_cls_here > OMNI_MAX_CLASSES) return cudaErrorInvalidValue;
  if (a.precision == OMNI_FP32) return head_t<float>(a, st);
  return a.precision == OMNI_FP16 ? head_t<__half>(a, st) : head_t<__nv_bfloat16>(a, st);
}

}  // namespace omni
