// Omni-Seg dynamic head (Sec. 2.2): the controller turns the tile's global
// average-pooled bottleneck feature plus one-hot class and scale codes into the
// 153 parameters of a per-tile, per-class 1x1 head 8 -> 8 -> 8 -> 1, which is
// applied at every pixel of the pre-head feature h0 = ReLU(Wh y0 + bh).
//
// One fused kernel: each block first evaluates the controller for its tile
// and every class of the scale (theta kept in shared memory), then runs the
// pre-head and all heads over 4096 pixels, writing FP32 logits.
#include "omni_internal.cuh"

namespace omni {
namespace {

constexpr int kHeadThreads = 256;
constexpr int kPixPerBlock = 4096;

template <typename T> __device__ __forceinline__ float ld(const T* p);
template <> __device__ __forceinline__ float ld<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <int C0, typename T>
__global__ void __launch_bounds__(kHeadThreads) k_head(HeadArgs a) {
  __shared__ float theta[OMNI_MAX_CLASSES][kHeadParams];
  __shared__ float wh[kHeadCh * C0], bh[kHeadCh];
  __shared__ float gs[1024];
  const int b = blockIdx.y;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int zdim = a.Cb + a.n_classes + a.n_scales;
  for (int i = t; i < kHeadCh * C0; i += kHeadThreads) wh[i] = a.wh[i];
  if (t < kHeadCh) bh[t] = a.bh[t];
  for (int i = t; i < a.Cb; i += kHeadThreads) gs[i] = a.g[(long long)b * a.Cb + i];
  __syncthreads();
  // controller: theta_c = Wc [g; onehot(c); onehot(scale)] + bc, one warp per row
  for (int row = warp; row < kHeadParams; row += kHeadThreads / 32) {
    const float* w = a.wc + (long long)row * zdim;
    float s = 0.f;
    for (int k = lane; k < a.Cb; k += 32) s = fmaf(w[k], gs[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      float common = s + w[a.Cb + a.n_classes + a.scale] + a.bc[row];
      for (int ci = 0; ci < a.n_cls_here; ++ci) theta[ci][row] = common + w[a.Cb + a.cls_ids[ci]];
    }
  }
  __syncthreads();

  const long long PP = (long long)a.P * a.P;
  const T* Y = static_cast<const T*>(a.y0) + (long long)b * PP * C0;
  float* out = a.logits + (long long)(a.slot0 + b) * a.n_cls_here * PP;
  const long long p0 = (long long)blockIdx.x * kPixPerBlock;
  for (int q = t; q < kPixPerBlock; q += kHeadThreads) {
    long long p = p0 + q;
    if (p >= PP) break;
    float y[C0];
#pragma unroll
    for (int c = 0; c < C0; ++c) y[c] = ld<T>(Y + p * C0 + c);
    float h0[kHeadCh];
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) {
      float s = bh[o];
#pragma unroll
      for (int c = 0; c < C0; ++c) s = fmaf(wh[o * C0 + c], y[c], s);
      h0[o] = fmaxf(s, 0.f);
    }
    for (int ci = 0; ci < a.n_cls_here; ++ci) {
      const float* th = theta[ci];
      float h1[kHeadCh], h2[kHeadCh];
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        float s = th[136 + o];
#pragma unroll
        for (int c = 0; c < kHeadCh; ++c) s = fmaf(th[o * 8 + c], h0[c], s);
        h1[o] = fmaxf(s, 0.f);
      }
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        float s = th[144 + o];
#pragma unroll
        for (int c = 0; c < kHeadCh; ++c) s = fmaf(th[64 + o * 8 + c], h1[c], s);
        h2[o] = fmaxf(s, 0.f);
      }
      float s = th[152];
#pragma unroll
      for (int c = 0; c < kHeadCh; ++c) s = fmaf(th[128 + c], h2[c], s);
      out[ci * PP + p] = s;
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

cudaError_t launch_head(const HeadArgs& a, cudaStream_t st) {
  if (a.Cb > 1024 || a.n_cls_here < 1 || a.n_cls_here > OMNI_MAX_CLASSES) return cudaErrorInvalidValue;
  return a.precision == OMNI_FP32 ? head_t<float>(a, st) : head_t<__nv_bfloat16>(a, st);
}

}  // namespace omni
