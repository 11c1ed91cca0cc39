// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "omniseg.h"

namespace omni {

constexpr int kThumb = 32;          // tissue thumbnail box (40x pixels)
constexpr int kHeadCh = 8;          // dynamic head width
constexpr int kHeadParams = 153;    // 8*8 + 8*8 + 8 + 8 + 8 + 1
constexpr int kMaxEll = 32;         // ellipses of the synthetic slide generator
constexpr int kMaxLevels = 6;

// Device-side error word bits (set by bounded waits, read by the host).
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBounds = 2u;

// ---------------------------------------------------------------- slide prep
struct SlideGeom {
  int H, W;              // slide
  int Hp, Wp, lead;      // padded 40x canvas and leading border
  int th, tw;            // thumbnail
  int n_scales;
  int factors[OMNI_MAX_SCALES];
  int gh[OMNI_MAX_SCALES], gw[OMNI_MAX_SCALES];
  int grid_off[OMNI_MAX_SCALES + 1];   // offsets of per-scale grids in the flag array
  int P;
  int S[OMNI_MAX_SCALES];             // tile stride of each scale, in its pixels
};

// k_slide.cu
cudaError_t launch_synth(const int64_t* ell_host, int n_ell, uint64_t seed, int structures, int slide_w,
                         int y0, int x0, int h, int w, uint8_t* out, int64_t stride, cudaStream_t st);
cudaError_t launch_pad(const uint8_t* rgb, int64_t stride, const SlideGeom& g, uint8_t* canvas,
                       cudaStream_t st);
// 40x canvas -> downsampled images for factors 2/4/8 (any may be null) + 8x8 block sums
cudaError_t launch_pyramid(const uint8_t* c40, int64_t stride40, int Hp, int Wp, uint8_t* c20,
                           uint8_t* c10, uint8_t* c5, uint16_t* blk8, cudaStream_t st);
cudaError_t launch_tissue(const uint16_t* blk8, const SlideGeom& g, int median_k, uint8_t* grey,
                          uint8_t* blurred, int32_t* hist, int32_t* otsu, uint8_t* mask,
                          cudaStream_t st);
// median blur, histogram, Otsu and mask from an existing thumbnail grey image
// Sec. 2.1 contour step: clears tissue regions (8-connected mask pixels) of
// fewer than min_area pixels.  region / area: th * tw int32 scratch each; err
// gets kErrTimeout if a union or find loop exceeds its bound.
cudaError_t launch_area_filter(uint8_t* mask, int th, int tw, int min_area, int32_t* region, int32_t* area,
                               unsigned* err, cudaStream_t st);
cudaError_t launch_tissue_grey(const uint8_t* grey, const SlideGeom& g, int median_k, uint8_t* blurred,
                               int32_t* hist, int32_t* otsu, uint8_t* mask, cudaStream_t st);
cudaError_t launch_tiles(const uint8_t* mask, const SlideGeom& g, int filter, int32_t* tiles,
                         int32_t* counts, uint8_t* flags, int32_t* slot_map, cudaStream_t st);

// ---------------------------------------------------------------- network
struct ConvLayerW {
  int cin, cout, cproj;          // cproj = channels of the residual projection (0: none)
  float* w_f32;                  // [9*cin][cout]   K-major rows for the FFMA path
  float* wp_f32;                 // [cproj][cout]
  __nv_bfloat16* w_bf16;         // [cout][9*cin]   K contiguous, for tcgen05
  __nv_bfloat16* wp_bf16;        // [cout][cproj]
  float* gamma;                  // [cout]
  float* beta;                   // [cout]
  // E4M3 experiment (cin, cout multiples of 128): rows [cout][9*cin] of
  // E4M3(w / s_w[o]) with s_w[o] = max |w[o]| / 448; null where not prepared
  uint8_t* w_e4m3;
  float* s_w;
};

enum ResMode { RES_NONE = 0, RES_TENSOR = 1, RES_RGB = 2 };

// Canvases the tiles of one network batch are read from: tile b's origin
// (tiles3[3 b + 1], tiles3[3 b + 2]) lies in canvas tiles3[3 b] (its slide in
// a multi-slide call, its scale in a one-slide call).  Every canvas is u8 RGB
// with its own row stride; rows are its height (for the TMA raw-window maps).
constexpr int kMaxCanvases = 16;
struct CanvasTab {
  const uint8_t* ptr[kMaxCanvases];
  long long stride[kMaxCanvases];
  int rows[kMaxCanvases];
};

struct ConvArgs {
  int B, R, cin, cout;
  const void* x; int x_cs, x_co;          // input NHWC (channel stride / offset)
  const void* r; int r_cs, r_co, cr;      // residual input for RES_TENSOR
  int res_mode;
  // RES_RGB / first layer: tiles read straight from the uint8 canvases; tile b
  // has origin (tiles3[3 b + 1], tiles3[3 b + 2]) in canvas cv.ptr[tiles3[3 b]]
  CanvasTab cv; const int32_t* tiles3;
  void* y; int y_cs, y_co;                // output NHWC
  ConvLayerW w;                           // device pointers, passed by value
  unsigned* err;
  // FP32 path only: raw = 1 writes the bare convolution sum to y (no norm, no
  // ReLU) and, with RES_TENSOR, the bare projection sum to y2 (channel stride
  // y2_cs); used by the backward's recomputation
  int raw;
  void* y2; int y2_cs;
  int f16;                                // tensor-core operands: 0 BF16, 1 FP16
  // Optional outputs fused into the epilogue of the small-N tensor-core
  // kernels (TcConfig kinds 1-4; see tc_fuses_pool / tc_fuses_head):
  // pool = 2x2 max-pool of y, NHWC [B][R/2][R/2] with channel stride pool_cs;
  // head_* = pre-head + dynamic heads of the tile (as launch_head), written as
  // FP32 logits [slot0 + b][head_ncls][R*R]; y may then be null (not stored).
  void* pool; int pool_cs;
  const float* head_theta;                // [B][head_ncls][153]
  const float* head_wh; const float* head_bh;   // [8][cout], [8]
  float* head_logits; int head_slot0, head_ncls;
};

// k_conv_f32.cu (plain FP32 path + precision-generic helpers)
cudaError_t launch_conv_first(const ConvArgs& a, int precision, cudaStream_t st);
cudaError_t launch_conv_f32(const ConvArgs& a, cudaStream_t st);
cudaError_t launch_maxpool(int precision, int B, int R, int C, const void* x, int x_cs, int x_co,
                           void* y, int y_cs, int y_co, cudaStream_t st);
// E4M3 experiment: max |x| of n BF16 values (float bits, atomicMax into a
// zeroed word) and x quantised to E4M3 bytes with one scale
cudaError_t launch_absmax_bf16(const void* x, long long n, unsigned* out_bits, cudaStream_t st);
cudaError_t launch_quant_e4m3(const void* x, long long n, float inv_scale, uint8_t* q, cudaStream_t st);
// the same inside the network, scale on the device: amax_bits (zeroed by the
// caller) receives max |x| over npix pixels of cin channels (channel stride
// x_cs, offset x_co), q the contiguous E4M3(x * 448 / max|x|), and
// gamma_out[o] = gamma[o] * s_w[o] * max|x| / 448
cudaError_t launch_e4m3_activation(const void* x, long long npix, int cin, int x_cs, int x_co,
                                   unsigned* amax_bits, uint8_t* q, const float* gamma, const float* s_w,
                                   int cout, float* gamma_out, cudaStream_t st);
cudaError_t launch_upsample(int precision, int B, int R, int C, const void* x, int x_cs,
                            int x_co, void* y, int y_cs, int y_co, cudaStream_t st);

// k_conv_tc.cu (BF16 tcgen05 implicit GEMM)
struct TcConfig {
  int kind;     // 0: per-tap A loads, 1: small-N variant (resident weights, 8x16 tiles),
                // 2: dx-in-N variant (horizontal taps stacked along N, lane-shuffle sum),
                // 3: small-N variant with two 8x16 blocks per tile (32-channel chunks),
                // 4: dx-in-N variant with two blocks per tile (cout 32),
                // 6: kind 3 on CTA pairs (cta_group::2 MMAs, M = 256),
                // 7: kind 4 once per 32-output-channel slice (cout 64..256),
                // 8: kind 0 on CTA pairs (N tile 128 / 256, 64-channel chunks)
  int bn;       // N tile
  int ck;       // channel chunk (32 -> 64-byte swizzle, 64 -> 128-byte swizzle)
  int stages;   // pipeline stages (small-N variant; per-tap derives its own)
};
cudaError_t launch_conv_tc(const ConvArgs& a, cudaStream_t st);
cudaError_t launch_conv_tc_cfg(const ConvArgs& a, const TcConfig& c, cudaStream_t st);
// E4M3 experiment: per-tap conv (TcConfig kind 0 or 8, N tile 128 / 256, chunk
// 128) on E4M3 activations (x) and weights (w.w_bf16 holding bytes), FP32
// accumulation, BF16 output; the dequantisation scales ride in w.gamma
cudaError_t launch_conv_tc_e4m3(const ConvArgs& a, const TcConfig& c, cudaStream_t st);
cudaError_t launch_conv_tc_cfg_bf16(const ConvArgs& a, const TcConfig& c, cudaStream_t st);
cudaError_t launch_conv_tc_cfg_f16(const ConvArgs& a, const TcConfig& c, cudaStream_t st);
int tc_candidates(int R, int cin, int cout, int cr, TcConfig* out, int max);
// first layer (cin = 3) on the tensor cores: operand rows gathered from the
// uint8 canvas; weights w.w_bf16 hold FP16 values [cout][32] (K = tap * 3 +
// channel, zero padded) in every precision; the output is the pipeline's type
bool conv_first_tc_supported(int R, int cout, const CanvasTab& cv);
cudaError_t launch_conv_first_tc(const ConvArgs& a, cudaStream_t st);
cudaError_t launch_conv_first_tc_bf16(const ConvArgs& a, cudaStream_t st);
cudaError_t launch_conv_first_tc_f16(const ConvArgs& a, cudaStream_t st);
// whether a configuration's epilogue computes ConvArgs::pool / the fused head
bool tc_fuses_pool(const TcConfig& c);
bool tc_fuses_head(const TcConfig& c, int cout, int ncls);
TcConfig tc_default(int R, int cin, int cout, int cr);
bool conv_tc_supported(int R, int cin, int cout, int cr);

// k_head.cu
struct HeadArgs {
  int B, P, C0, Cb, n_classes, n_scales, scale;
  int n_cls_here; int cls_ids[OMNI_MAX_CLASSES];
  const void* y0; int precision;           // [B][P][P][C0]
  const float* g;                          // [B][Cb]
  const float* wh; const float* bh;        // [8][C0], [8]
  const float* wc; const float* bc;        // [153][Cb + ncls + nscl], [153]
  int slot0;                               // output slot of tile 0 (tile b -> slot0 + b)
  float* logits;                           // [slot][n_cls_here][P*P]
  float* theta;                            // [B][n_cls_here][153] controller output
  const void* bott; int Rb;                // bottleneck [B][Rb][Rb][Cb] (fused GAP + controller)
  float* gap_out;                          // [B][Cb] GAP written by the fused kernel (or null)
};
// GAP of the bottleneck and the controller in one launch: per tile the mean of
// every bottleneck channel, then theta for every class of the scale
cudaError_t launch_gap_controller(const HeadArgs& a, cudaStream_t st);
// pre-head + dynamic heads over every pixel, reading theta
cudaError_t launch_head(const HeadArgs& a, cudaStream_t st);

// k_stitch.cu
struct StitchArgs {
  int hs, ws;                 // canvas size at this scale
  int oy0, ox0, oh, ow;       // output crop window in canvas pixels
  int P, S, gh, gw, f;
  const int32_t* slot_map;    // [gh][gw] index of the tile in the scale's foreground list, or -1
  const float* logits;        // [slot][n_cls][P*P]; slot = (index + slot_base) mod slot_cap (0: no ring)
  int slot_cap;
  int slot_base;              // added to the slot map's index before the ring modulo
  int row0, nrows;            // output rows row0 .. row0 + nrows - 1 (a band of the crop)
  int n_cls; int cls_ids[OMNI_MAX_CLASSES];
  int mode;                   // OMNI_STITCH_*
  const float* window;        // [P] separable overlap-average weight t(u); null = flat
  const uint8_t* tissue; int th, tw;   // thumbnail mask (null: no AND)
  uint8_t* labels[OMNI_MAX_CLASSES];
  float* out_logits[OMNI_MAX_CLASSES];
  uint16_t* coverage;
  uint8_t* argmax;
};
cudaError_t launch_stitch(const StitchArgs& a, cudaStream_t st);

// k_backward.cu
struct NPix { long long n[OMNI_MAX_CLASSES]; };
struct BwdHeadArgs {
  int B, P, ci, n_cls;                     // tiles in the batch, tile size, class index in scale list
  const float* theta;                      // [B][n_cls][153]
  const float *wh, *bh, *g2, *b2;          // pre-head, last block's second norm
  const int32_t* tiles3;                   // tile origins (scale pixels)
  int oy0, ox0, oh, ow;                    // label-map crop of this scale
  const uint16_t* cov;                     // [oh][ow] coverage
  const float* dL;                         // [oh][ow] dloss / dstitched logit of class ci
  const float *c2, *pr;                    // [B*P*P][C0] bare second conv and projection sums
  float* dh0;                              // [B*P*P][8]
  float* dtheta_partial;                   // [B][n_cls][blocks][153]
  float *y0, *dh0_pre, *dy0_pre, *dc2;     // pre-head backward outputs
};
int loss_blocks();
cudaError_t launch_loss_partial(const float* L, const uint8_t* gt, long long n, float* partial,
                                cudaStream_t st);
cudaError_t launch_loss_final(const float* partial, int n_cls, const NPix& npix, float* sums,
                              float* loss, cudaStream_t st);
cudaError_t launch_loss_grad(const float* L, const uint8_t* gt, long long n, const float* sums, float npix,
                             int n_cls, float* dL, cudaStream_t st);
cudaError_t launch_affine_relu(const float* c, const float* g, const float* b, int C, long long n, float* a,
                               cudaStream_t st);
cudaError_t launch_relu_bwd(const float* da, const float* c1, const float* g1, const float* b1, int C,
                            long long n, float* da_pre, float* dc, cudaStream_t st);
int head_bwd_blocks(int P);
cudaError_t launch_head_bwd(const BwdHeadArgs& a, int C0, cudaStream_t st);
cudaError_t launch_prehead_bwd(const BwdHeadArgs& a, int C0, long long npx, cudaStream_t st);
int wgrad_chunks(long long npx);
cudaError_t launch_wgrad(const float* dY, int O, const float* X, int x_cs, int cin, int taps, int P,
                         long long npx, float* partial, float2* acc, cudaStream_t st);
cudaError_t launch_colsum(const float* A, const float* B, int C, long long npx, float* partial, float2* acc,
                          cudaStream_t st);
cudaError_t launch_ctrl_bwd(const float* dtheta_partial, int hblocks, int B, int n_cls, const int* cls_ids_dev,
                            int n_classes, int n_scales, int scale, const float* g, int Cb, float2* dwc,
                            float2* dbc, cudaStream_t st);
cudaError_t launch_to_f32(const float2* a, long long n, float* out, cudaStream_t st);

}  // namespace omni
