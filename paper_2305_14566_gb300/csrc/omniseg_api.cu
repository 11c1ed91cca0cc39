// C ABI of the library (declared in omniseg.h): context, weights layout,
// workspace planning and the orchestration of the three stages of the
// whole-slide pipeline (Sec. 2.1 tiling, Sec. 2.2 segmentation, Sec. 2.3
// aggregation).
#include <cuda_fp8.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "omni_internal.cuh"

using namespace omni;

struct omni_ctx {
  omni_config cfg;
  std::string err;
  int device = 0;
  bool have_weights = false;
  void* wdev = nullptr;
  std::vector<ConvLayerW> enc1, enc2, dec1, dec2;   // indexed by level
  ConvLayerW dec2t0{};                              // last block's second conv, transposed + flipped
  float *wh = nullptr, *bh = nullptr, *wc = nullptr, *bc = nullptr;
  unsigned* d_err = nullptr;
  float* d_window = nullptr;                        // [P] overlap-average weight t(u), or null (flat)
  int32_t* h_counts = nullptr;                      // pinned
  uint8_t* h_flags = nullptr;                       // pinned copy of the tile flags (band stitching)
  size_t h_flags_n = 0;
  // host-buffer calls: each stitched band's labels go to the host on copy_st
  // while the network runs on (host_labels[c] non-null for the classes wanted)
  uint8_t* const* host_labels = nullptr;
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> band_ev;
  size_t band_ev_used = 0;

  // timing
  bool timing = false;
  struct Ev { cudaEvent_t a, b; int kind, tag; double work; };
  std::vector<Ev> evs;
  size_t ev_used = 0;
  double work[4] = {0, 0, 0, 0};
  int64_t launches = 0;
  int64_t tiles_done = 0;
  // conv autotuner: layer shape -> fastest tensor-core configuration
  bool autotune = false;
  int force_kind = -1;         // >= 0: every layer with a candidate of this kind runs it
  // E4M3 experiment: eligible convs run on E4M3 operands (omni_set_e4m3);
  // e8 is their scratch (quantised activation, max |x|, scaled gamma)
  bool e4m3 = false;
  uint8_t* e8 = nullptr;
  size_t e8_bytes = 0;
  std::map<std::array<int, 6>, TcConfig> tuned;
  // CUDA graph of the post-tiling launch chain (network + stitch)
  bool graphs = false;
  bool fuse = true;            // epilogue fusion of max-pool and head
  std::vector<uint64_t> last_key, graph_key;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0, graph_tiles = 0;
  double graph_stitch_bytes = 0;
  bool capturing = false;
};

namespace {

omni_status fail(omni_ctx* c, omni_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

// next event of the context's pool (timing disabled), created on demand
cudaError_t band_event(omni_ctx* c, cudaEvent_t* out) {
  if (c->band_ev_used == c->band_ev.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    c->band_ev.push_back(e);
  }
  *out = c->band_ev[c->band_ev_used++];
  return cudaSuccess;
}

// Forget the captured launch chain: its kernel arguments hold device pointers
// (weights) and kernel choices (fusion, autotuned configurations) of the state
// it was captured in, so any change to that state must drop it.
void drop_graph(omni_ctx* c) {
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  c->last_key.clear();
  c->graph_key.clear();
}

omni_status cuda_fail(omni_ctx* c, cudaError_t e, const char* where) {
  return fail(c, OMNI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define OMNI_CU(expr, where)                                   \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);   \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr size_t kNone = ~size_t(0);   // offset of a workspace region that is absent
size_t take(size_t& off, size_t bytes) {
  size_t o = align_up(off, 256);
  off = o + bytes;
  return o;
}

int widths(const omni_config& c, int l) { return c.base << l; }

// Tile stride of scale s in its own pixels (Sec. 3.2 strides the 40x scale by
// 256 and the 10x and 5x scales by 64); 0 in scale_stride means `stride`.
int stride_of(const omni_config& c, int s) { return c.scale_stride[s] > 0 ? c.scale_stride[s] : c.stride; }

// The padded canvas is a whole number of every scale's stride (f_s * S_s 40x
// pixels), hence of 32-pixel thumbnail cells: lcm over the scales.
long long canvas_unit(const omni_config& c) {
  long long u = 1;
  for (int s = 0; s < c.n_scales; ++s) {
    long long v = (long long)c.factors[s] * stride_of(c, s), a = u, b = v;
    while (b) { long long t = a % b; a = b; b = t; }
    u = u / a * v;
    if (u > (1LL << 30)) return u;
  }
  return u;
}

std::string validate(const omni_config& c) {
  if (c.levels < 2 || c.levels > kMaxLevels) return "levels must be in 2..6";
  if (c.base < 8 || c.base > 64 || c.base % 8) return "base must be 8, 16, 32 or 64";
  if (c.patch <= 0 || c.patch % (1 << (c.levels - 1)) || (c.patch >> (c.levels - 1)) < 2)
    return "patch must be divisible by 2^(levels-1) with a bottleneck of at least 2x2";
  if (c.stride <= 0 || c.patch % c.stride || c.stride % 4) return "stride must divide patch and be a multiple of 4";
  if (c.n_scales < 1 || c.n_scales > OMNI_MAX_SCALES) return "n_scales must be 1..4";
  int fmax = 1;
  for (int s = 0; s < c.n_scales; ++s) {
    int f = c.factors[s];
    if (f != 1 && f != 2 && f != 4 && f != 8) return "factors must be 1, 2, 4 or 8";
    for (int q = 0; q < s; ++q)
      if (c.factors[q] == f) return "factors must be distinct";
    fmax = std::max(fmax, f);
    const int st = stride_of(c, s);
    if (c.scale_stride[s] < 0 || c.patch % st || st % 4)
      return "every scale stride must divide patch and be a multiple of 4";
    if ((f * st) % kThumb) return "factor times stride must be a multiple of 32 at every scale";
  }
  if (canvas_unit(c) > (1 << 20)) return "the lcm of factor times stride over the scales is too large";
  if (c.n_classes < 1 || c.n_classes > OMNI_MAX_CLASSES) return "n_classes must be 1..16";
  for (int k = 0; k < c.n_classes; ++k)
    if (c.class_scale[k] < 0 || c.class_scale[k] >= c.n_scales) return "class_scale out of range";
  if (c.precision != OMNI_FP32 && c.precision != OMNI_BF16 && c.precision != OMNI_FP16)
    return "precision must be FP32, BF16 or FP16";
  if (c.stitch_mode != OMNI_STITCH_AVG && c.stitch_mode != OMNI_STITCH_VOTE) return "bad stitch_mode";
  if (c.stitch_window < OMNI_WINDOW_FLAT || c.stitch_window > OMNI_WINDOW_HANN) return "bad stitch_window";
  if (c.median_k < 1 || c.median_k % 2 == 0 || c.median_k > 255) return "median_k must be odd, 1..255";
  if (c.min_tissue_area < 0) return "min_tissue_area must be >= 0";
  if (c.max_batch < 1 || c.max_batch > 4096) return "max_batch must be 1..4096";
  if (c.pad_lead < 0 || c.pad_lead % fmax) return "pad_lead must be a non-negative multiple of the largest factor";
  if (widths(c, c.levels - 1) > 1024) return "bottleneck wider than 1024 channels";
  return "";
}

int fmax_of(const omni_config& c) {
  int f = 1;
  for (int s = 0; s < c.n_scales; ++s) f = std::max(f, c.factors[s]);
  return f;
}

struct Plan {
  SlideGeom g;
  bool pad;
  int ncls_s[OMNI_MAX_SCALES];
  int cap[OMNI_MAX_SCALES];   // tile-logit ring slots per scale (a multiple of max_batch)
  // tile stage
  size_t canvas, c20, c10, c5, blk8, grey, blur, hist, otsu, mask, tiles, counts, flags, slot;
  size_t region, area;               // tissue-region labels and sizes (area filter)
  size_t tile_end;
  // network stage
  size_t logits, tmp, pooled, pooled2, cat[kMaxLevels], bott, ydec[kMaxLevels], gap, theta;
  size_t net_end;
  // host-buffer variant
  size_t in, lab[OMNI_MAX_CLASSES];
  size_t total;
  uint64_t flops_per_tile;
};

bool make_plan(const omni_config& c, int H, int W, Plan& p) {
  if (H <= 0 || W <= 0) return false;
  memset(&p, 0, sizeof(p));
  const int fmax = fmax_of(c);
  const long long unit = canvas_unit(c);
  const long long minimum = (fmax * (long long)c.patch + unit - 1) / unit * unit;
  auto ext = [&](long long d) {
    long long v = (d + 2LL * c.pad_lead + unit - 1) / unit * unit;
    return std::max<long long>(v, minimum);
  };
  SlideGeom& g = p.g;
  g.H = H; g.W = W; g.lead = c.pad_lead;
  long long Hp = ext(H), Wp = ext(W);
  if (Hp > (1LL << 30) || Wp > (1LL << 30)) return false;
  g.Hp = (int)Hp; g.Wp = (int)Wp;
  g.th = g.Hp / kThumb; g.tw = g.Wp / kThumb;
  g.n_scales = c.n_scales; g.P = c.patch;
  g.grid_off[0] = 0;
  for (int s = 0; s < c.n_scales; ++s) {
    int f = c.factors[s];
    g.factors[s] = f;
    g.S[s] = stride_of(c, s);
    g.gh[s] = (g.Hp / f - c.patch) / g.S[s] + 1;
    g.gw[s] = (g.Wp / f - c.patch) / g.S[s] + 1;
    g.grid_off[s + 1] = g.grid_off[s] + g.gh[s] * g.gw[s];
    p.ncls_s[s] = 0;
  }
  for (int k = 0; k < c.n_classes; ++k) p.ncls_s[c.class_scale[k]]++;
  p.pad = (g.Hp != H) || (g.Wp != W) || c.pad_lead != 0;
  bool has[9] = {false};
  for (int s = 0; s < c.n_scales; ++s) has[c.factors[s]] = true;
  size_t off = 0;
  const size_t HpWp = (size_t)g.Hp * g.Wp;
  p.canvas = p.pad ? take(off, HpWp * 3) : kNone;
  p.c20 = has[2] ? take(off, HpWp / 4 * 3) : kNone;
  p.c10 = has[4] ? take(off, HpWp / 16 * 3) : kNone;
  p.c5 = has[8] ? take(off, HpWp / 64 * 3) : kNone;
  p.blk8 = take(off, HpWp / 64 * 3 * sizeof(uint16_t));
  size_t tn = (size_t)g.th * g.tw;
  p.grey = take(off, tn);
  p.blur = take(off, tn);
  p.mask = take(off, tn);
  p.hist = take(off, 256 * 4);
  p.otsu = take(off, 4);
  p.region = c.min_tissue_area > 0 ? take(off, tn * 4) : kNone;
  p.area = c.min_tissue_area > 0 ? take(off, tn * 4) : kNone;
  int ntile = g.grid_off[c.n_scales];
  p.tiles = take(off, (size_t)ntile * 3 * 4);
  p.counts = take(off, (OMNI_MAX_SCALES + 1) * 4);
  p.flags = take(off, (size_t)ntile);
  p.slot = take(off, (size_t)ntile * 4);
  p.tile_end = align_up(off, 256);

  const size_t e = c.precision == OMNI_FP32 ? 4 : 2;
  const size_t B = (size_t)c.max_batch;
  const size_t PP = (size_t)c.patch * c.patch;
  // Tile logits live in a ring: an output band of S rows is stitched once the
  // P/S tile rows covering it are done, so at any time the ring holds at most
  // P/S tile rows that a band still needs, the row being filled and one batch;
  // (P/S + 1) rows + a batch, rounded to whole batches so a batch's slots
  // never wrap.  The logit memory no longer grows with the slide's height.
  size_t lmax = 0;
  for (int s = 0; s < c.n_scales; ++s) {
    const long long rows = (c.patch + g.S[s] - 1) / g.S[s] + 1;
    long long cap = rows * g.gw[s] + (long long)B;
    cap = std::min<long long>(cap, (long long)g.gh[s] * g.gw[s] + (long long)B);
    cap = (cap + (long long)B - 1) / (long long)B * (long long)B;
    p.cap[s] = (int)cap;
    lmax = std::max(lmax, (size_t)cap * (size_t)p.ncls_s[s]);
  }
  p.logits = take(off, lmax * PP * 4);
  const int L = c.levels;
  p.tmp = take(off, B * PP * widths(c, 0) * e);
  // pooled encoder inputs ping-pong between two buffers (level l reads buffer
  // (l-1) % 2 while its second conv's epilogue may write the next level's
  // pooled input into the other): level 1's input is the larger
  p.pooled = take(off, B * PP / 4 * widths(c, 0) * e);
  p.pooled2 = take(off, B * PP / 16 * widths(c, std::min(1, L - 1)) * e);
  for (int l = 0; l < L - 1; ++l) {
    size_t R = (size_t)(c.patch >> l);
    p.cat[l] = take(off, B * R * R * 3 * widths(c, l) * e);
    p.ydec[l] = take(off, B * R * R * widths(c, l) * e);
  }
  size_t Rb = (size_t)(c.patch >> (L - 1));
  p.bott = take(off, B * Rb * Rb * widths(c, L - 1) * e);
  p.gap = take(off, B * widths(c, L - 1) * 4);
  p.theta = take(off, B * OMNI_MAX_CLASSES * kHeadParams * 4);
  p.net_end = align_up(off, 256);
  p.in = take(off, (size_t)H * W * 3);
  for (int k = 0; k < c.n_classes; ++k) {
    int f = c.factors[c.class_scale[k]];
    p.lab[k] = take(off, (size_t)((H + f - 1) / f) * ((W + f - 1) / f));
  }
  p.total = align_up(off, 256);

  // algorithmic conv FLOPs of one tile (2 per multiply-add)
  double fl = 0;
  for (int l = 0; l < L; ++l) {
    double R2 = (double)(c.patch >> l) * (c.patch >> l);
    double cin = l == 0 ? 3 : widths(c, l - 1), co = widths(c, l);
    fl += 2 * R2 * co * (9 * cin + 9 * co + cin);
  }
  for (int l = 0; l < L - 1; ++l) {
    double R2 = (double)(c.patch >> l) * (c.patch >> l);
    double co = widths(c, l), cin = 3 * co;
    fl += 2 * R2 * co * (9 * cin + 9 * co + cin);
  }
  p.flops_per_tile = (uint64_t)fl;
  return true;
}

// ------------------------------------------------------------------ bf16 (round to nearest even)
uint16_t to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

uint16_t to_fp16(float f) {
  const __half h = __float2half_rn(f);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
}

float fp16_value(uint16_t u) {
  __half h;
  memcpy(&h, &u, 2);
  return __half2float(h);
}

// 16-bit operand bits of the tensor-core path (BF16 or FP16)
uint16_t to_lp(float f, bool f16) { return f16 ? to_fp16(f) : to_bf16(f); }

// ------------------------------------------------------------------ timing helpers
struct Rec {
  omni_ctx* c;
  cudaStream_t st;
  int idx;
  // kind: 0 conv, 1 stitch, 2 head/GAP, 3 other; tag identifies the layer
  // (see omni_get_launch_times); work = algorithmic FLOPs (convs) or bytes
  Rec(omni_ctx* c_, cudaStream_t st_, int kind, int tag = -1, double work = 0)
      : c(c_), st(st_), idx(-1) {
    if (!c->timing) return;
    if (c->ev_used == c->evs.size()) {
      omni_ctx::Ev e{};
      cudaEventCreate(&e.a);
      cudaEventCreate(&e.b);
      c->evs.push_back(e);
    }
    idx = (int)c->ev_used++;
    c->evs[idx].kind = kind;
    c->evs[idx].tag = tag;
    c->evs[idx].work = work;
    cudaEventRecord(c->evs[idx].a, st);
  }
  ~Rec() {
    if (idx >= 0) cudaEventRecord(c->evs[idx].b, st);
  }
};

}  // namespace

// ====================================================================== C ABI
extern "C" {

omni_status omni_create(const omni_config* cfg, omni_ctx** out) {
  if (!cfg || !out) return OMNI_EINVAL;
  *out = nullptr;
  std::string v = validate(*cfg);
  if (!v.empty()) {
    static thread_local std::string last;
    last = v;
    fprintf(stderr, "omni_create: %s\n", v.c_str());
    return OMNI_EINVAL;
  }
  omni_ctx* ctx = new omni_ctx();
  ctx->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counts, OMNI_MAX_SLIDES * (OMNI_MAX_SCALES + 1) * sizeof(int32_t));
  if (e == cudaSuccess && cfg->stitch_window != OMNI_WINDOW_FLAT) {
    // one-dimensional weight of the stitch window, from its definition
    const int P = cfg->patch;
    std::vector<float> t(P);
    for (int u = 0; u < P; ++u) {
      if (cfg->stitch_window == OMNI_WINDOW_TENT) {
        t[u] = (float)std::min(u + 1, P - u);
      } else {
        const double sn = std::sin(M_PI * (u + 0.5) / P);
        t[u] = (float)(sn * sn);
      }
    }
    e = cudaMalloc(&ctx->d_window, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_window, t.data(), P * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "omni_create: %s\n", cudaGetErrorString(e));
    omni_destroy(ctx);
    return OMNI_ECUDA;
  }
  *out = ctx;
  return OMNI_OK;
}

void omni_destroy(omni_ctx* ctx) {
  if (!ctx) return;
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->wdev) cudaFree(ctx->wdev);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_window) cudaFree(ctx->d_window);
  if (ctx->e8) cudaFree(ctx->e8);
  if (ctx->h_counts) cudaFreeHost(ctx->h_counts);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  for (cudaEvent_t e : ctx->band_ev) cudaEventDestroy(e);
  if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
  for (auto& e : ctx->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  delete ctx;
}

const char* omni_last_error(const omni_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t omni_weights_count(const omni_config* cfg) {
  if (!cfg || !validate(*cfg).empty()) return -1;
  const omni_config& c = *cfg;
  int64_t n = 0;
  auto block = [&](int64_t cin, int64_t co) { n += co * cin * 9 + 2 * co + co * co * 9 + 2 * co + co * cin; };
  for (int l = 0; l < c.levels; ++l) block(l == 0 ? 3 : widths(c, l - 1), widths(c, l));
  for (int l = c.levels - 2; l >= 0; --l) block(3 * widths(c, l), widths(c, l));
  n += kHeadCh * widths(c, 0) + kHeadCh;
  int64_t zdim = widths(c, c.levels - 1) + c.n_classes + c.n_scales;
  n += kHeadParams * zdim + kHeadParams;
  return n;
}

omni_status omni_load_weights(omni_ctx* ctx, const float* blob, int64_t n_floats) {
  if (!ctx || !blob) return fail(ctx, OMNI_EINVAL, "null argument");
  const omni_config& c = ctx->cfg;
  const bool f16 = c.precision == OMNI_FP16;
  int64_t need = omni_weights_count(&c);
  if (n_floats != need)
    return fail(ctx, OMNI_EWEIGHTS, "weights blob has " + std::to_string(n_floats) +
                                         " floats, configuration needs " + std::to_string(need));
  for (int64_t i = 0; i < n_floats; ++i)
    if (!std::isfinite(blob[i])) return fail(ctx, OMNI_EWEIGHTS, "non-finite weight at " + std::to_string(i));

  // host staging of every device array, 256-byte aligned
  std::vector<uint8_t> host;
  size_t off = 0;
  auto alloc = [&](size_t bytes) {
    size_t o = take(off, bytes);
    if (host.size() < off) host.resize(off + (1 << 20));
    return o;
  };
  struct Pending { size_t w32, wp32, w16, wp16, g, b, w8, s8; int cin, cout, cproj; bool has8; };
  std::vector<Pending> pend;
  const float* src = blob;
  auto conv = [&](int cin, int cout, int cproj_blob, int cproj_used) {
    // blob: w1-style [cout][cin][3][3], g, b ; projection handled by caller
    Pending q{};
    q.cin = cin; q.cout = cout; q.cproj = cproj_used;
    // 16-bit weights: [cout][9 cin] (tap-major K).  The first layer's rows are
    // FP16 in every precision, padded to K = 32 for its tensor-core kernel,
    // and carry the input normalisation and the layer's norm: its operands are
    // A = 512 + u per colour byte u (639.5 at a padding tap), and v = 2u/255 - 1
    // = (A - 639.5) 2/255, so K entries 0..26 hold W = g[o] w 2/255 (rounded)
    // and entries 27, 28 (operands 1) the FP16 pair hi + lo of
    // B = b[o] - 639.5 sum_k W_k, summed over the rounded W: the MMA yields
    // g * conv(v) + b with only the weights' rounding
    const size_t kdim = cin == 3 ? 32 : (size_t)9 * cin;
    q.w32 = alloc((size_t)9 * cin * cout * 4);
    q.w16 = alloc(kdim * cout * 2);
    q.g = alloc((size_t)cout * 4);
    q.b = alloc((size_t)cout * 4);
    float* w32 = reinterpret_cast<float*>(host.data() + q.w32);
    uint16_t* w16 = reinterpret_cast<uint16_t*>(host.data() + q.w16);
    const float* gsrc = src + (size_t)cout * cin * 9;     // the layer's norm scale and shift
    const float* bsrc = gsrc + cout;
    for (int o = 0; o < cout; ++o) {
      double wsum = 0.0;                                 // first layer: sum of the stored W
      for (int ci = 0; ci < cin; ++ci)
        for (int tap = 0; tap < 9; ++tap) {
          float v = src[((size_t)o * cin + ci) * 9 + tap];
          w32[((size_t)tap * cin + ci) * cout + o] = v;
          uint16_t h;
          if (cin == 3) {
            h = to_fp16((float)((double)gsrc[o] * v * (2.0 / 255.0)));
            wsum += (double)fp16_value(h);
          } else {
            h = to_lp(v, f16);
          }
          w16[(size_t)o * kdim + (size_t)tap * cin + ci] = h;
        }
      if (cin == 3) {
        const double shift = (double)bsrc[o] - 639.5 * wsum;
        const uint16_t hi = to_fp16((float)shift);
        w16[(size_t)o * kdim + 27] = hi;
        w16[(size_t)o * kdim + 28] = to_fp16((float)(shift - (double)fp16_value(hi)));
        for (int k = 29; k < 32; ++k) w16[(size_t)o * kdim + k] = 0;
      }
    }
    if (cin % 128 == 0 && cout % 128 == 0) {
      // E4M3 rows for the experiment: per-row scale s_w = max |w[o]| / 448
      q.has8 = true;
      q.w8 = alloc(kdim * cout);
      q.s8 = alloc((size_t)cout * 4);
      uint8_t* w8 = host.data() + q.w8;
      float* s8 = reinterpret_cast<float*>(host.data() + q.s8);
      for (int o = 0; o < cout; ++o) {
        float m = 0.f;
        for (size_t k = 0; k < kdim; ++k) m = std::max(m, std::fabs(src[(size_t)o * kdim + k]));
        const double sw = m > 0.f ? (double)m / 448.0 : 1.0;
        for (int ci = 0; ci < cin; ++ci)
          for (int tap = 0; tap < 9; ++tap)
            w8[(size_t)o * kdim + (size_t)tap * cin + ci] = __nv_cvt_float_to_fp8(
                (float)(src[((size_t)o * cin + ci) * 9 + tap] / sw), __NV_SATFINITE, __NV_E4M3);
        s8[o] = (float)sw;
      }
    }
    src += (size_t)cout * cin * 9;
    memcpy(host.data() + q.g, src, cout * 4);
    src += cout;
    memcpy(host.data() + q.b, src, cout * 4);
    src += cout;
    (void)cproj_blob;
    return q;
  };
  auto proj = [&](Pending& q, int cproj) {
    q.wp32 = alloc((size_t)cproj * q.cout * 4);
    q.wp16 = alloc((size_t)cproj * q.cout * 2);
    float* wp32 = reinterpret_cast<float*>(host.data() + q.wp32);
    uint16_t* wp16 = reinterpret_cast<uint16_t*>(host.data() + q.wp16);
    for (int o = 0; o < q.cout; ++o)
      for (int ci = 0; ci < cproj; ++ci) {
        float v = src[(size_t)o * cproj + ci];
        wp32[(size_t)ci * q.cout + o] = v;
        wp16[(size_t)o * cproj + ci] = to_lp(v, f16);
      }
    src += (size_t)q.cout * cproj;
    q.cproj = cproj;
  };
  const int L = c.levels;
  std::vector<Pending> e1(L), e2(L), d1(L), d2(L);
  for (int l = 0; l < L; ++l) {
    int cin = l == 0 ? 3 : widths(c, l - 1), co = widths(c, l);
    e1[l] = conv(cin, co, 0, 0);
    e2[l] = conv(co, co, cin, cin);
    proj(e2[l], cin);
  }
  for (int l = L - 2; l >= 0; --l) {
    int co = widths(c, l), cin = 3 * co;
    d1[l] = conv(cin, co, 0, 0);
    d2[l] = conv(co, co, cin, cin);
    proj(d2[l], cin);
  }
  // dec0 conv2 transposed and flipped (input gradient of the last block):
  // wt[(tap * C0 + o)][ci] = w2[o][ci][8 - tap]
  const int C0 = widths(c, 0);
  const size_t o_w2t = alloc((size_t)9 * C0 * C0 * 4);
  {
    const float* w2 = src - ((size_t)C0 * C0 * 9 + 2 * C0 + (size_t)C0 * 3 * C0);  // dec0.w2 in the blob
    float* wt = reinterpret_cast<float*>(host.data() + o_w2t);
    for (int o = 0; o < C0; ++o)
      for (int ci = 0; ci < C0; ++ci)
        for (int tap = 0; tap < 9; ++tap)
          wt[((size_t)tap * C0 + o) * C0 + ci] = w2[((size_t)o * C0 + ci) * 9 + (8 - tap)];
  }
  size_t o_wh = alloc((size_t)kHeadCh * widths(c, 0) * 4);
  memcpy(host.data() + o_wh, src, (size_t)kHeadCh * widths(c, 0) * 4);
  src += kHeadCh * widths(c, 0);
  size_t o_bh = alloc(kHeadCh * 4);
  memcpy(host.data() + o_bh, src, kHeadCh * 4);
  src += kHeadCh;
  size_t zdim = widths(c, L - 1) + c.n_classes + c.n_scales;
  size_t o_wc = alloc((size_t)kHeadParams * zdim * 4);
  memcpy(host.data() + o_wc, src, (size_t)kHeadParams * zdim * 4);
  src += kHeadParams * zdim;
  size_t o_bc = alloc(kHeadParams * 4);
  memcpy(host.data() + o_bc, src, kHeadParams * 4);
  src += kHeadParams;
  if (src - blob != n_floats) return fail(ctx, OMNI_EWEIGHTS, "internal blob walk mismatch");

  size_t total = align_up(off, 256);
  host.resize(total);
  void* dev = nullptr;
  OMNI_CU(cudaMalloc(&dev, total), "cudaMalloc(weights)");
  cudaError_t e = cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(ctx, e, "cudaMemcpy(weights)");
  }
  drop_graph(ctx);     // the captured chain still points at the old weights
  if (ctx->wdev) cudaFree(ctx->wdev);
  ctx->wdev = dev;
  uint8_t* d = static_cast<uint8_t*>(dev);
  auto mk = [&](const Pending& q) {
    ConvLayerW w{};
    w.cin = q.cin; w.cout = q.cout; w.cproj = q.cproj;
    w.w_f32 = reinterpret_cast<float*>(d + q.w32);
    w.w_bf16 = reinterpret_cast<__nv_bfloat16*>(d + q.w16);
    w.gamma = reinterpret_cast<float*>(d + q.g);
    w.beta = reinterpret_cast<float*>(d + q.b);
    if (q.cproj) {
      w.wp_f32 = reinterpret_cast<float*>(d + q.wp32);
      w.wp_bf16 = reinterpret_cast<__nv_bfloat16*>(d + q.wp16);
    }
    if (q.has8) {
      w.w_e4m3 = d + q.w8;
      w.s_w = reinterpret_cast<float*>(d + q.s8);
    }
    return w;
  };
  ctx->enc1.assign(L, {}); ctx->enc2.assign(L, {}); ctx->dec1.assign(L, {}); ctx->dec2.assign(L, {});
  for (int l = 0; l < L; ++l) { ctx->enc1[l] = mk(e1[l]); ctx->enc2[l] = mk(e2[l]); }
  for (int l = 0; l < L - 1; ++l) { ctx->dec1[l] = mk(d1[l]); ctx->dec2[l] = mk(d2[l]); }
  ctx->dec2t0 = ctx->dec2[0];
  ctx->dec2t0.w_f32 = reinterpret_cast<float*>(d + o_w2t);
  ctx->dec2t0.cproj = 0;
  ctx->wh = reinterpret_cast<float*>(d + o_wh);
  ctx->bh = reinterpret_cast<float*>(d + o_bh);
  ctx->wc = reinterpret_cast<float*>(d + o_wc);
  ctx->bc = reinterpret_cast<float*>(d + o_bc);
  ctx->have_weights = true;
  return OMNI_OK;
}

omni_status omni_query(const omni_config* cfg, int32_t H, int32_t W, omni_sizes* out) {
  if (!cfg || !out || !validate(*cfg).empty()) return OMNI_EINVAL;
  Plan p;
  if (!make_plan(*cfg, H, W, p)) return OMNI_EINVAL;
  memset(out, 0, sizeof(*out));
  out->Hp = p.g.Hp; out->Wp = p.g.Wp; out->thumb_h = p.g.th; out->thumb_w = p.g.tw;
  for (int s = 0; s < cfg->n_scales; ++s) {
    out->grid_h[s] = p.g.gh[s];
    out->grid_w[s] = p.g.gw[s];
    int f = cfg->factors[s];
    out->out_h[s] = (H + f - 1) / f;
    out->out_w[s] = (W + f - 1) / f;
  }
  out->n_tiles_max = p.g.grid_off[cfg->n_scales];
  out->tile_workspace_bytes = p.tile_end;
  out->workspace_bytes = p.total;
  out->flops_per_tile = p.flops_per_tile;
  return OMNI_OK;
}

}  // extern "C"

namespace {

struct Prep {
  const uint8_t* c[OMNI_MAX_SCALES];
  int64_t cs[OMNI_MAX_SCALES];
  int ch[OMNI_MAX_SCALES];      // canvas rows
};

// canvas table of a one-slide batch: the tiles' first field is their scale s,
// so every entry is that scale's canvas
CanvasTab one_canvas(const Prep& pr, int s) {
  CanvasTab t{};
  for (int k = 0; k < kMaxCanvases; ++k) {
    t.ptr[k] = pr.c[s];
    t.stride[k] = pr.cs[s];
    t.rows[k] = pr.ch[s];
  }
  return t;
}

// Sec. 2.1 stages on the device; fills `pr` with every scale's canvas.
omni_status run_prep(omni_ctx* ctx, const uint8_t* rgb, int64_t stride, const Plan& p, uint8_t* ws,
                     cudaStream_t st, Prep& pr) {
  const omni_config& c = ctx->cfg;
  const SlideGeom& g = p.g;
  const uint8_t* c40 = rgb;
  int64_t s40 = stride;
  if (p.pad) {
    Rec r(ctx, st, 3, 700);
    OMNI_CU(launch_pad(rgb, stride, g, ws + p.canvas, st), "pad");
    ctx->launches++;
    c40 = ws + p.canvas;
    s40 = (int64_t)g.Wp * 3;
  } else if ((stride % 8) || (reinterpret_cast<uintptr_t>(rgb) % 8)) {
    return fail(ctx, OMNI_EINVAL, "unpadded slides need 8-byte aligned rows");
  }
  uint8_t* c20 = p.c20 != kNone ? ws + p.c20 : nullptr;
  uint8_t* c10 = p.c10 != kNone ? ws + p.c10 : nullptr;
  uint8_t* c5 = p.c5 != kNone ? ws + p.c5 : nullptr;
  {
    Rec r(ctx, st, 3, 701);
    OMNI_CU(launch_pyramid(c40, s40, g.Hp, g.Wp, c20, c10, c5, (uint16_t*)(ws + p.blk8), st), "pyramid");
    ctx->launches++;
  }
  for (int s = 0; s < c.n_scales; ++s) {
    int f = c.factors[s];
    pr.c[s] = f == 1 ? c40 : f == 2 ? c20 : f == 4 ? c10 : c5;
    pr.cs[s] = f == 1 ? s40 : (int64_t)(g.Wp / f) * 3;
    pr.ch[s] = g.Hp / f;
    if (!pr.c[s]) return fail(ctx, OMNI_EINVAL, "internal: no canvas for scale " + std::to_string(s));
  }
  {
    Rec r(ctx, st, 3, 702);
    OMNI_CU(launch_tissue((uint16_t*)(ws + p.blk8), g, c.median_k, ws + p.grey, ws + p.blur,
                          (int32_t*)(ws + p.hist), (int32_t*)(ws + p.otsu), ws + p.mask, st),
            "tissue");
    ctx->launches += 5;
    if (c.min_tissue_area > 0) {
      OMNI_CU(launch_area_filter(ws + p.mask, g.th, g.tw, c.min_tissue_area, (int32_t*)(ws + p.region),
                                 (int32_t*)(ws + p.area), ctx->d_err, st),
              "area filter");
      ctx->launches += 4;
    }
  }
  {
    Rec r(ctx, st, 3, 703);
    OMNI_CU(launch_tiles(ws + p.mask, g, c.tissue_filter, (int32_t*)(ws + p.tiles),
                         (int32_t*)(ws + p.counts), ws + p.flags, (int32_t*)(ws + p.slot), st),
            "tiles");
    ctx->launches += 2;
  }
  return OMNI_OK;
}

double conv_flops(const ConvArgs& a) {
  const double cr = a.res_mode == RES_TENSOR ? a.cr : (a.res_mode == RES_RGB ? 3 : 0);
  return 2.0 * a.B * a.R * a.R * a.cout * (9.0 * a.cin + cr);
}

// Times every legal tensor-core configuration of a layer on the real operands
// (two warm-up launches, then three timed with events) and returns the
// fastest; the launches only rewrite the layer's own output.  Synchronises.
// the launch arguments for configuration c: fused outputs it cannot compute
// are dropped (the caller then runs the separate kernels); with the head
// fused, the block output itself is not stored
ConvArgs fit_fused(const ConvArgs& in, const TcConfig& c) {
  ConvArgs a = in;
  if (!tc_fuses_pool(c)) a.pool = nullptr;
  if (a.head_theta && tc_fuses_head(c, a.cout, a.head_ncls)) a.y = nullptr;
  else a.head_theta = nullptr;
  return a;
}

// device time of one separate head launch (for the autotuner's comparison);
// it writes the batch's logit slots, which the real launch later overwrites
float time_head(omni_ctx* ctx, const HeadArgs& h, cudaStream_t st) {
  cudaEvent_t e0, e1;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess) return 0.f;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 0.f; }
  bool ok = launch_head(h, st) == cudaSuccess && cudaEventRecord(e0, st) == cudaSuccess;
  for (int r = 0; r < 3 && ok; ++r) ok = launch_head(h, st) == cudaSuccess;
  ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
       cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->launches += 4;
  return ok ? ms / 3.f : 0.f;
}

// Times every candidate configuration on the real operands and keeps the
// fastest.  unfused_ms is added to candidates that cannot compute the
// requested fused head, which then needs its own kernel (measured by the caller).
TcConfig tune_conv(omni_ctx* ctx, const ConvArgs& a, cudaStream_t st, float unfused_ms = 0.f) {
  const int cr = a.res_mode == RES_TENSOR ? a.cr : 0;
  TcConfig cands[16];
  const int n = tc_candidates(a.R, a.cin, a.cout, cr, cands, 16);
  TcConfig best = tc_default(a.R, a.cin, a.cout, cr);
  float best_ms = 1e30f;
  // a layer that carries the fused head keeps it whenever some variant can
  // compute it: the dynamic head then never needs a launch of its own
  bool head_only = false;
  for (int i = 0; i < n && a.head_theta; ++i) head_only |= tc_fuses_head(cands[i], a.cout, a.head_ncls);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return best;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return best; }
  // a variant that cannot fuse a requested 2x2 max-pool pays the separate
  // pooling launch (the conv's output is pooled afterwards)
  float pool_ms = 0.f;
  if (a.pool && a.y) {
    bool ok = launch_maxpool(ctx->cfg.precision, a.B, a.R, a.cout, a.y, a.y_cs, a.y_co, a.pool, a.pool_cs, 0,
                             st) == cudaSuccess &&
              cudaEventRecord(e0, st) == cudaSuccess;
    for (int r = 0; r < 3 && ok; ++r)
      ok = launch_maxpool(ctx->cfg.precision, a.B, a.R, a.cout, a.y, a.y_cs, a.y_co, a.pool, a.pool_cs, 0, st) ==
           cudaSuccess;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(&pool_ms, e0, e1) == cudaSuccess;
    pool_ms = ok ? pool_ms / 3.f : 0.f;
    ctx->launches += 4;
  }
  for (int i = 0; i < n; ++i) {
    if (head_only && !tc_fuses_head(cands[i], a.cout, a.head_ncls)) continue;
    const ConvArgs ai = fit_fused(a, cands[i]);
    bool ok = launch_conv_tc_cfg(ai, cands[i], st) == cudaSuccess &&
              launch_conv_tc_cfg(ai, cands[i], st) == cudaSuccess;
    ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
    for (int r = 0; r < 3 && ok; ++r) ok = launch_conv_tc_cfg(ai, cands[i], st) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (a.head_theta && !ai.head_theta) ms += 3.f * unfused_ms;   // three timed launches
    if (a.pool && !ai.pool) ms += 3.f * pool_ms;
    if (ok && ms < best_ms) {
      best_ms = ms;
      best = cands[i];
    }
    ctx->launches += 5;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// run one conv layer; the fused pool / head requested in `in` run only where
// the chosen kernel supports them, and *pooled / *headed report whether they did
omni_status run_conv(omni_ctx* ctx, const ConvArgs& in, cudaStream_t st, int tag, bool* pooled = nullptr,
                     bool* headed = nullptr, const HeadArgs* head = nullptr) {
  Rec r(ctx, st, 0, tag, conv_flops(in));
  ConvArgs a = in;
  cudaError_t e;
  int nlaunch = 1;
  if (ctx->cfg.precision == OMNI_FP32) {
    a.pool = nullptr;
    a.head_theta = nullptr;
    e = launch_conv_f32(a, st);
  } else {
    if (!conv_tc_supported(a.R, a.cin, a.cout, a.res_mode == RES_TENSOR ? a.cr : 0))
      return fail(ctx, OMNI_EINVAL, "BF16 tensor-core conv does not support R=" + std::to_string(a.R) +
                                        " cin=" + std::to_string(a.cin) + " cout=" + std::to_string(a.cout));
    const int cr = a.res_mode == RES_TENSOR ? a.cr : 0;
    if (ctx->e4m3 && a.res_mode == RES_NONE && !a.pool && !a.head_theta && a.y && a.w.w_e4m3 &&
        a.cout <= 512 && (a.R == 16 || a.R == 32 || a.R == 64 || a.R % 128 == 0)) {
      // E4M3 experiment: quantise this call's activation with its own scale
      const long long npix = (long long)a.B * a.R * a.R;
      const size_t need = (size_t)npix * a.cin + 4096;
      if (ctx->e8_bytes < need) {
        if (ctx->e8) cudaFree(ctx->e8);
        ctx->e8 = nullptr;
        ctx->e8_bytes = 0;
        OMNI_CU(cudaMalloc(&ctx->e8, need), "E4M3 scratch");
        ctx->e8_bytes = need;
      }
      unsigned* amax = reinterpret_cast<unsigned*>(ctx->e8);
      float* gq = reinterpret_cast<float*>(ctx->e8 + 256);
      uint8_t* q = ctx->e8 + 4096;
      OMNI_CU(cudaMemsetAsync(amax, 0, 4, st), "E4M3 max");
      OMNI_CU(launch_e4m3_activation(a.x, npix, a.cin, a.x_cs, a.x_co, amax, q, a.w.gamma, a.w.s_w, a.cout, gq, st),
              "E4M3 activation");
      ConvArgs a8 = a;
      a8.x = q; a8.x_cs = a.cin; a8.x_co = 0;
      a8.w.w_bf16 = reinterpret_cast<__nv_bfloat16*>(a.w.w_e4m3);
      a8.w.gamma = gq;
      const TcConfig c8{(long long)a.R * a.R % 256 == 0 ? 8 : 0, a.cout % 256 == 0 ? 256 : 128, 128, 0};
      e = launch_conv_tc_e4m3(a8, c8, st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "conv (E4M3)");
      ctx->launches += 4;
      if (pooled) *pooled = false;
      if (headed) *headed = false;
      return OMNI_OK;
    }
    TcConfig cfg = tc_default(a.R, a.cin, a.cout, cr);
    if (ctx->force_kind >= 0) {
      // the first candidate of the forced kind (its largest chunk first), if the
      // shape has one and it can take this layer's fused head
      TcConfig cands[16];
      const int n = tc_candidates(a.R, a.cin, a.cout, cr, cands, 16);
      // (the CTA-pair kernel needs an even count of 16 x 16 tiles)
      const bool pair_ok = ((long long)a.B * (a.R / 16) * (a.R / 16)) % 2 == 0;
      for (int i = 0; i < n; ++i)
        if (cands[i].kind == ctx->force_kind && (cands[i].kind != 6 || pair_ok) &&
            (!a.head_theta || tc_fuses_head(cands[i], a.cout, a.head_ncls) || !tc_fuses_head(cfg, a.cout, a.head_ncls))) {
          cfg = cands[i];
          break;
        }
      ctx->tuned[std::array<int, 6>{a.R, a.cin, a.cout, cr, a.res_mode, a.B}] = cfg;   // reported by omni_get_tuned
    } else if (ctx->autotune) {
      const std::array<int, 6> key{a.R, a.cin, a.cout, cr, a.res_mode, a.B};
      auto it = ctx->tuned.find(key);
      if (it != ctx->tuned.end()) {
        cfg = it->second;
      } else if (!ctx->capturing) {
        float head_ms = 0.f;
        if (a.head_theta && head) head_ms = time_head(ctx, *head, st);
        cfg = tune_conv(ctx, a, st, head_ms);
        ctx->tuned[key] = cfg;
      }
    }
    a = fit_fused(in, cfg);
    e = launch_conv_tc_cfg(a, cfg, st);
    if (cfg.kind == 7) nlaunch = a.cout / 32;      // one launch per 32-channel slice
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "conv");
  ctx->launches += nlaunch;
  if (pooled) *pooled = a.pool != nullptr;
  if (headed) *headed = a.head_theta != nullptr;
  return OMNI_OK;
}

// U-Net + heads for `nb` tiles of one scale.
omni_status run_batch(omni_ctx* ctx, const Plan& p, uint8_t* ws, int s, const CanvasTab& cv,
                      const int32_t* tiles3, int nb, int slot0, int ncls,
                      const int* cls, cudaStream_t st, bool stop_before_dec0 = false) {
  const omni_config& c = ctx->cfg;
  const int L = c.levels, prec = c.precision;
  auto C = [&](int l) { return widths(c, l); };
  void* tmp = ws + p.tmp;
  void* pool_buf[2] = {ws + p.pooled, ws + p.pooled2};
  void* bott = ws + p.bott;
  ConvArgs base{};
  base.B = nb;
  base.cv = cv;
  base.tiles3 = tiles3;
  base.err = ctx->d_err;
  base.f16 = c.precision == OMNI_FP16 ? 1 : 0;
  // encoder output location of level l
  auto enc_out = [&](int l, void*& ptr, int& cs, int& co) {
    if (l < L - 1) { ptr = ws + p.cat[l]; cs = 3 * C(l); co = 2 * C(l); }
    else { ptr = bott; cs = C(l); co = 0; }
  };
  {
    ConvArgs a = base;
    a.R = c.patch; a.cin = 3; a.cout = C(0);
    a.y = tmp; a.y_cs = C(0); a.y_co = 0;
    a.w = ctx->enc1[0];
    Rec r(ctx, st, 0, 0, conv_flops(a));
    cudaError_t e = prec != OMNI_FP32 && conv_first_tc_supported(a.R, a.cout, cv)
                        ? launch_conv_first_tc(a, st)
                        : launch_conv_first(a, prec, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "conv_first");
    ctx->launches++;
  }
  // pooled_done: the previous level's second conv wrote the pooled input
  bool pooled_done = false;
  {
    ConvArgs a = base;
    a.R = c.patch; a.cin = C(0); a.cout = C(0);
    a.x = tmp; a.x_cs = C(0); a.x_co = 0;
    a.res_mode = RES_RGB; a.cr = 3;
    enc_out(0, a.y, a.y_cs, a.y_co);
    a.w = ctx->enc2[0];
    if (L > 1 && ctx->fuse) { a.pool = pool_buf[0]; a.pool_cs = C(0); }
    omni_status r = run_conv(ctx, a, st, 1, &pooled_done);
    if (r) return r;
  }
  for (int l = 1; l < L; ++l) {
    const int R = c.patch >> l;
    void* pooled = pool_buf[(l - 1) & 1];
    void* pp; int pcs, pco;
    enc_out(l - 1, pp, pcs, pco);
    if (!pooled_done) {
      Rec r(ctx, st, 3, 200 + l);
      OMNI_CU(launch_maxpool(prec, nb, 2 * R, C(l - 1), pp, pcs, pco, pooled, C(l - 1), 0, st), "maxpool");
      ctx->launches++;
    }
    ConvArgs a = base;
    a.R = R; a.cin = C(l - 1); a.cout = C(l);
    a.x = pooled; a.x_cs = C(l - 1); a.x_co = 0;
    a.y = tmp; a.y_cs = C(l); a.y_co = 0;
    a.w = ctx->enc1[l];
    omni_status r = run_conv(ctx, a, st, 10 * l);
    if (r) return r;
    ConvArgs b2 = base;
    b2.R = R; b2.cin = C(l); b2.cout = C(l);
    b2.x = tmp; b2.x_cs = C(l); b2.x_co = 0;
    b2.res_mode = RES_TENSOR; b2.r = pooled; b2.r_cs = C(l - 1); b2.r_co = 0; b2.cr = C(l - 1);
    enc_out(l, b2.y, b2.y_cs, b2.y_co);
    b2.w = ctx->enc2[l];
    if (l < L - 1 && ctx->fuse) { b2.pool = pool_buf[l & 1]; b2.pool_cs = C(l); }
    pooled_done = false;
    r = run_conv(ctx, b2, st, 10 * l + 1, &pooled_done);
    if (r) return r;
  }
  float* gap = reinterpret_cast<float*>(ws + p.gap);
  HeadArgs h{};
  h.B = nb; h.P = c.patch; h.C0 = C(0); h.Cb = C(L - 1);
  h.n_classes = c.n_classes; h.n_scales = c.n_scales; h.scale = s;
  h.n_cls_here = ncls;
  for (int k = 0; k < ncls; ++k) h.cls_ids[k] = cls[k];
  h.precision = prec; h.g = gap;
  h.wh = ctx->wh; h.bh = ctx->bh; h.wc = ctx->wc; h.bc = ctx->bc;
  h.slot0 = slot0;
  h.logits = reinterpret_cast<float*>(ws + p.logits);
  h.theta = reinterpret_cast<float*>(ws + p.theta);
  h.bott = bott; h.Rb = c.patch >> (L - 1); h.gap_out = gap;
  {
    // GAP of the bottleneck and the controller of every class of the scale
    Rec r(ctx, st, 2, 401);
    OMNI_CU(launch_gap_controller(h, st), "gap + controller");
    ctx->launches++;
  }
  const void* y = bott;
  int y_cs = C(L - 1);
  bool head_done = false;   // the last decoder conv ran the pre-head and heads in its epilogue
  for (int l = L - 2; l >= 0; --l) {
    const int R = c.patch >> l;
    void* cat = ws + p.cat[l];
    {
      Rec r(ctx, st, 3, 300 + l);
      OMNI_CU(launch_upsample(prec, nb, R, 2 * C(l), y, y_cs, 0, cat, 3 * C(l), 0, st), "upsample");
      ctx->launches++;
    }
    if (l == 0 && stop_before_dec0) return OMNI_OK;
    ConvArgs a = base;
    a.R = R; a.cin = 3 * C(l); a.cout = C(l);
    a.x = cat; a.x_cs = 3 * C(l); a.x_co = 0;
    a.y = tmp; a.y_cs = C(l); a.y_co = 0;
    a.w = ctx->dec1[l];
    omni_status r = run_conv(ctx, a, st, 100 + 10 * l);
    if (r) return r;
    ConvArgs b2 = base;
    b2.R = R; b2.cin = C(l); b2.cout = C(l);
    b2.x = tmp; b2.x_cs = C(l); b2.x_co = 0;
    b2.res_mode = RES_TENSOR; b2.r = cat; b2.r_cs = 3 * C(l); b2.r_co = 0; b2.cr = 3 * C(l);
    b2.y = ws + p.ydec[l]; b2.y_cs = C(l); b2.y_co = 0;
    b2.w = ctx->dec2[l];
    if (l == 0 && ctx->fuse) {
      b2.head_theta = h.theta; b2.head_wh = h.wh; b2.head_bh = h.bh;
      b2.head_logits = h.logits; b2.head_slot0 = h.slot0; b2.head_ncls = h.n_cls_here;
    }
    HeadArgs h_here = h;
    h_here.y0 = ws + p.ydec[0];
    r = run_conv(ctx, b2, st, 100 + 10 * l + 1, nullptr, l == 0 ? &head_done : nullptr, l == 0 ? &h_here : nullptr);
    if (r) return r;
    y = ws + p.ydec[l];
    y_cs = C(l);
  }
  if (!head_done) {
    h.y0 = y;
    Rec r(ctx, st, 2, 500);
    OMNI_CU(launch_head(h, st), "head");
    ctx->launches++;
  }
  return OMNI_OK;
}

// Band stitching of one slide at one scale.  Output block row k (canvas rows
// k S .. k S + S - 1) is covered by tile rows k - P/S + 1 .. k, so it is final
// once tile rows 0..k are done; advance() takes the number of this slide's
// tiles (of this scale) done so far and stitches every block row that became
// final.  A band's labels are also queued for the host when the call has host
// outputs.
struct Bands {
  StitchArgs a;
  int s = 0, S = 1, nblk = 0, next_blk = 0, row_ptr = 0, gh = 0;
  const int* row_end = nullptr;
  const int* cls = nullptr;
  int ncls = 0;

  omni_status stitch_to(omni_ctx* ctx, int blk_end, cudaStream_t st) {
    if (blk_end <= next_blk) return OMNI_OK;
    const int y0 = std::max(0, next_blk * S - a.oy0), y1 = std::min(a.oh, blk_end * S - a.oy0);
    next_blk = blk_end;
    if (y1 <= y0) return OMNI_OK;
    a.row0 = y0;
    a.nrows = y1 - y0;
    {
      Rec rr(ctx, st, 1, 600 + s);
      OMNI_CU(launch_stitch(a, st), "stitch");
      ctx->launches++;
    }
    if (ctx->host_labels) {
      // the band is final: its label rows go to the host while the next batches run
      cudaEvent_t ev;
      OMNI_CU(band_event(ctx, &ev), "band event");
      OMNI_CU(cudaEventRecord(ev, st), "band event record");
      OMNI_CU(cudaStreamWaitEvent(ctx->copy_st, ev, 0), "band wait");
      for (int k = 0; k < ncls; ++k) {
        uint8_t* dst = ctx->host_labels[cls[k]];
        if (!dst || !a.labels[k]) continue;
        const size_t o0 = (size_t)y0 * a.ow, nb = (size_t)(y1 - y0) * a.ow;
        OMNI_CU(cudaMemcpyAsync(dst + o0, a.labels[k] + o0, nb, cudaMemcpyDeviceToHost, ctx->copy_st),
                "download band");
      }
    }
    return OMNI_OK;
  }
  omni_status advance(omni_ctx* ctx, int done, cudaStream_t st) {
    while (row_ptr < gh && row_end[row_ptr] <= done) ++row_ptr;
    return stitch_to(ctx, row_ptr == gh ? nblk : row_ptr, st);
  }
  omni_status finish(omni_ctx* ctx, cudaStream_t st) { return stitch_to(ctx, nblk, st); }
};

// Stitch state of one slide (plan p, tile stage at ws_prep) at scale s; the
// slide's tile logits sit in the ring at (index + slot_base) mod cap.
Bands make_bands(omni_ctx* ctx, const omni_config& c, const Plan& p, const uint8_t* ws_prep, const uint8_t* ws_net,
                 const Plan& pn, const omni_outputs* out, int H, int W, int s, const int* cls, int ncls, int n_s,
                 int slot_base, const std::vector<int>& row_end, double& stitch_bytes) {
  Bands b;
  const int f = c.factors[s];
  StitchArgs& a = b.a;
  a = StitchArgs{};
  a.hs = p.g.Hp / f; a.ws = p.g.Wp / f;
  a.oy0 = c.pad_lead / f; a.ox0 = c.pad_lead / f;
  a.oh = (H + f - 1) / f; a.ow = (W + f - 1) / f;
  a.window = ctx->d_window; a.P = c.patch; a.S = p.g.S[s]; a.gh = p.g.gh[s]; a.gw = p.g.gw[s]; a.f = f;
  a.slot_map = reinterpret_cast<const int32_t*>(ws_prep + p.slot) + p.g.grid_off[s];
  a.slot_cap = pn.cap[s];
  a.slot_base = slot_base;
  a.logits = reinterpret_cast<const float*>(ws_net + pn.logits);
  a.n_cls = ncls;
  for (int k = 0; k < ncls; ++k) {
    a.cls_ids[k] = cls[k];
    a.labels[k] = out->labels[cls[k]];
    a.out_logits[k] = out->logits[cls[k]];
  }
  a.mode = c.stitch_mode;
  a.tissue = c.tissue_and ? ws_prep + p.mask : nullptr;
  a.th = p.g.th; a.tw = p.g.tw;
  a.coverage = out->coverage[s];
  a.argmax = out->argmax[s];
  const double px = (double)a.oh * a.ow;
  stitch_bytes += (double)n_s * ncls * c.patch * c.patch * 4.0;
  for (int k = 0; k < ncls; ++k) stitch_bytes += px * ((a.labels[k] ? 1 : 0) + (a.out_logits[k] ? 4 : 0));
  stitch_bytes += px * ((a.coverage ? 2 : 0) + (a.argmax ? 1 : 0));
  b.s = s;
  b.S = p.g.S[s];
  b.nblk = a.hs / b.S;
  b.gh = p.g.gh[s];
  b.row_end = row_end.data();
  b.cls = cls;
  b.ncls = ncls;
  return b;
}

// classes of scale s selected by class_mask
int classes_at(const omni_config& c, int s, uint32_t class_mask, int* cls) {
  int n = 0;
  for (int k = 0; k < c.n_classes; ++k)
    if (c.class_scale[k] == s && (class_mask >> k & 1u)) cls[n++] = k;
  return n;
}

// the caller's stream waits for the last band copy (this also joins the copy
// stream back into a stream capture)
omni_status join_copies(omni_ctx* ctx, cudaStream_t st) {
  if (!ctx->host_labels) return OMNI_OK;
  cudaEvent_t ev;
  OMNI_CU(band_event(ctx, &ev), "band event");
  OMNI_CU(cudaEventRecord(ev, ctx->copy_st), "copy join record");
  OMNI_CU(cudaStreamWaitEvent(st, ev, 0), "copy join");
  return OMNI_OK;
}

// Everything after tiling: every batch of every requested scale, then the
// stitch + labels of each scale, band by band.  Launch-only (no
// synchronisation), so it can be captured into a CUDA graph.
omni_status run_network(omni_ctx* ctx, const omni_config& c, const Plan& p, uint8_t* ws, const Prep& pr,
                        const omni_outputs* out, int H, int W, uint32_t scale_mask, uint32_t class_mask,
                        const std::vector<std::vector<int>>& row_end, cudaStream_t st, double& stitch_bytes) {
  omni_status r = OMNI_OK;
  const int32_t* tiles = reinterpret_cast<const int32_t*>(ws + p.tiles);
  int toff = 0;
  for (int s = 0; s < c.n_scales; ++s) {
    const int n_s = ctx->h_counts[1 + s];
    int cls[OMNI_MAX_CLASSES];
    const int ncls = classes_at(c, s, class_mask, cls);
    if ((scale_mask >> s & 1u) && ncls > 0) {
      Bands b = make_bands(ctx, c, p, ws, ws, p, out, H, W, s, cls, ncls, n_s, 0, row_end[s], stitch_bytes);
      const int cap = p.cap[s];
      for (int start = 0; start < n_s; start += c.max_batch) {
        int nb = std::min(c.max_batch, n_s - start);
        r = run_batch(ctx, p, ws, s, one_canvas(pr, s), tiles + 3 * (toff + start), nb, start % cap, ncls,
                      cls, st);
        if (r) return r;
        r = b.advance(ctx, start + nb, st);
        if (r) return r;
      }
      r = b.finish(ctx, st);
      if (r) return r;
      ctx->tiles_done += n_s;
    }
    toff += n_s;
  }
  return join_copies(ctx, st);
}

// Runs the launch chain `chain(stitch_bytes)` eagerly, or, with graphs on and
// a capturable stream, captures it into the context's CUDA graph on the
// second call with the same key and replays that graph on later calls.
template <typename F>
omni_status run_graphed(omni_ctx* ctx, const std::vector<uint64_t>& key, cudaStream_t st, double& stitch_bytes,
                        F&& chain) {
  // the legacy default stream cannot be captured: such calls run eagerly
  const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
  // (the E4M3 experiment may allocate its scratch mid-chain: no capture)
  const bool use_graph = ctx->graphs && !ctx->timing && capturable && !ctx->e4m3;
  if (use_graph && ctx->graph_exec && key == ctx->graph_key) {
    OMNI_CU(cudaGraphLaunch(ctx->graph_exec, st), "graph launch");
    ctx->launches += ctx->graph_launches;
    ctx->tiles_done = ctx->graph_tiles;
    stitch_bytes = ctx->graph_stitch_bytes;
    return OMNI_OK;
  }
  if (use_graph && key == ctx->last_key) {
    // second call with the same geometry and buffers: capture and replay from now on
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    const int64_t before = ctx->launches;
    OMNI_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    ctx->capturing = true;
    omni_status r = chain(stitch_bytes);
    ctx->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (r) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      ctx->graph_exec = nullptr;
      return cuda_fail(ctx, ie, "graph instantiate");
    }
    ctx->graph_key = key;
    ctx->graph_launches = ctx->launches - before;
    ctx->graph_tiles = ctx->tiles_done;
    ctx->graph_stitch_bytes = stitch_bytes;
    OMNI_CU(cudaGraphLaunch(ctx->graph_exec, st), "graph launch");
    return OMNI_OK;
  }
  ctx->last_key = key;
  return chain(stitch_bytes);
}

omni_status check_ws(omni_ctx* ctx, void* ws, uint64_t bytes, uint64_t need) {
  if (!ws) return fail(ctx, OMNI_EINVAL, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(ctx, OMNI_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < need)
    return fail(ctx, OMNI_ENOMEM, "workspace has " + std::to_string(bytes) + " bytes, needs " + std::to_string(need));
  return OMNI_OK;
}

}  // namespace

extern "C" {

omni_status omni_tile_slide(omni_ctx* ctx, const uint8_t* rgb, int32_t H, int32_t W, int64_t stride,
                            void* ws_, uint64_t ws_bytes, const omni_tile_list* out, void* stream) {
  (void)cudaGetLastError();   // errors of earlier, unrelated calls are not ours to report
  if (!ctx || !rgb || !out || !out->tiles || !out->counts) return fail(ctx, OMNI_EINVAL, "null argument");
  if (stride < (int64_t)W * 3) return fail(ctx, OMNI_EINVAL, "row_stride < 3 W");
  Plan p;
  if (!make_plan(ctx->cfg, H, W, p)) return fail(ctx, OMNI_EINVAL, "bad slide size");
  omni_status r = check_ws(ctx, ws_, ws_bytes, p.tile_end);
  if (r) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  Prep pr;
  ctx->launches = 0;
  r = run_prep(ctx, rgb, stride, p, ws, st, pr);
  if (r) return r;
  const int n = p.g.grid_off[ctx->cfg.n_scales];
  OMNI_CU(cudaMemcpyAsync(out->tiles, ws + p.tiles, (size_t)n * 12, cudaMemcpyDeviceToDevice, st), "copy tiles");
  OMNI_CU(cudaMemcpyAsync(out->counts, ws + p.counts, (size_t)(1 + ctx->cfg.n_scales) * 4,
                          cudaMemcpyDeviceToDevice, st), "copy counts");
  if (out->flags) OMNI_CU(cudaMemcpyAsync(out->flags, ws + p.flags, n, cudaMemcpyDeviceToDevice, st), "copy flags");
  if (out->tissue)
    OMNI_CU(cudaMemcpyAsync(out->tissue, ws + p.mask, (size_t)p.g.th * p.g.tw, cudaMemcpyDeviceToDevice, st), "copy mask");
  if (out->otsu) OMNI_CU(cudaMemcpyAsync(out->otsu, ws + p.otsu, 4, cudaMemcpyDeviceToDevice, st), "copy otsu");
  return OMNI_OK;
}

omni_status omni_segment_slide(omni_ctx* ctx, const uint8_t* rgb, int32_t H, int32_t W, int64_t stride,
                               uint32_t scale_mask, uint32_t class_mask, void* ws_, uint64_t ws_bytes,
                               const omni_outputs* out, void* stream) {
  (void)cudaGetLastError();   // errors of earlier, unrelated calls are not ours to report
  if (!ctx || !rgb || !out) return fail(ctx, OMNI_EINVAL, "null argument");
  if (!ctx->have_weights) return fail(ctx, OMNI_ESTATE, "omni_load_weights has not been called");
  if (stride < (int64_t)W * 3) return fail(ctx, OMNI_EINVAL, "row_stride < 3 W");
  const omni_config& c = ctx->cfg;
  Plan p;
  if (!make_plan(c, H, W, p)) return fail(ctx, OMNI_EINVAL, "bad slide size");
  omni_status r = check_ws(ctx, ws_, ws_bytes, p.net_end);
  if (r) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  ctx->launches = 0;
  ctx->tiles_done = 0;
  ctx->band_ev_used = 0;
  Prep pr;
  r = run_prep(ctx, rgb, stride, p, ws, st, pr);
  if (r) return r;
  OMNI_CU(cudaMemcpyAsync(ctx->h_counts, ws + p.counts, (size_t)(1 + c.n_scales) * 4, cudaMemcpyDeviceToHost, st),
          "read tile counts");
  const size_t nflags = (size_t)p.g.grid_off[c.n_scales];
  if (ctx->h_flags_n < nflags) {
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    ctx->h_flags = nullptr;
    ctx->h_flags_n = 0;
    OMNI_CU(cudaMallocHost(&ctx->h_flags, nflags), "pinned tile flags");
    ctx->h_flags_n = nflags;
  }
  OMNI_CU(cudaMemcpyAsync(ctx->h_flags, ws + p.flags, nflags, cudaMemcpyDeviceToHost, st), "read tile flags");
  OMNI_CU(cudaStreamSynchronize(st), "sync after tiling");
  unsigned herr = 0;
  OMNI_CU(cudaMemcpy(&herr, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
  if (herr) return fail(ctx, OMNI_ETIMEOUT, "a device-side wait gave up in an earlier call");
  // foreground tiles in rows 0..i of every scale's grid: the band schedule of the stitch
  std::vector<std::vector<int>> row_end(c.n_scales);
  for (int s = 0; s < c.n_scales; ++s) {
    const uint8_t* fl = ctx->h_flags + p.g.grid_off[s];
    int acc = 0;
    row_end[s].resize(p.g.gh[s]);
    for (int i = 0; i < p.g.gh[s]; ++i) {
      for (int j = 0; j < p.g.gw[s]; ++j) acc += fl[(size_t)i * p.g.gw[s] + j] ? 1 : 0;
      row_end[s][i] = acc;
    }
  }

  // ---------------------------------------------------------------- network + stitch
  std::vector<uint64_t> key = {reinterpret_cast<uint64_t>(rgb), (uint64_t)H, (uint64_t)W, (uint64_t)stride,
                               scale_mask, class_mask, reinterpret_cast<uint64_t>(ws_),
                               reinterpret_cast<uint64_t>(st)};
  for (int s = 0; s <= c.n_scales; ++s) key.push_back((uint64_t)ctx->h_counts[s]);
  for (int s = 0; s < c.n_scales; ++s)
    for (int v : row_end[s]) key.push_back((uint64_t)v);
  for (int k = 0; k < OMNI_MAX_CLASSES; ++k) {
    key.push_back(reinterpret_cast<uint64_t>(out->labels[k]));
    key.push_back(reinterpret_cast<uint64_t>(out->logits[k]));
  }
  for (int s = 0; s < OMNI_MAX_SCALES; ++s) {
    key.push_back(reinterpret_cast<uint64_t>(out->coverage[s]));
    key.push_back(reinterpret_cast<uint64_t>(out->argmax[s]));
  }
  for (int k = 0; k < OMNI_MAX_CLASSES; ++k)
    key.push_back(reinterpret_cast<uint64_t>(ctx->host_labels ? ctx->host_labels[k] : nullptr));
  double stitch_bytes = 0;
  r = run_graphed(ctx, key, st, stitch_bytes, [&](double& sb) {
    return run_network(ctx, c, p, ws, pr, out, H, W, scale_mask, class_mask, row_end, st, sb);
  });
  if (r) return r;
  ctx->work[0] += (double)ctx->tiles_done * (double)p.flops_per_tile;
  ctx->work[1] += stitch_bytes;
  return OMNI_OK;
}

omni_status omni_segment_slide_host(omni_ctx* ctx, const uint8_t* rgb_host, int32_t H, int32_t W,
                                    int64_t stride, uint32_t scale_mask, uint32_t class_mask, void* ws_,
                                    uint64_t ws_bytes, uint8_t* const* labels_host, void* stream) {
  if (!ctx || !rgb_host || !labels_host) return fail(ctx, OMNI_EINVAL, "null argument");
  const omni_config& c = ctx->cfg;
  Plan p;
  if (!make_plan(c, H, W, p)) return fail(ctx, OMNI_EINVAL, "bad slide size");
  omni_status r = check_ws(ctx, ws_, ws_bytes, p.total);
  if (r) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  const int64_t dstride = (int64_t)W * 3;
  // packed rows go up as one linear copy; padded rows as a pitched copy
  if (stride == dstride)
    OMNI_CU(cudaMemcpyAsync(ws + p.in, rgb_host, (size_t)dstride * H, cudaMemcpyHostToDevice, st), "upload slide");
  else
    OMNI_CU(cudaMemcpy2DAsync(ws + p.in, dstride, rgb_host, stride, dstride, H, cudaMemcpyHostToDevice, st),
            "upload slide");
  omni_outputs o{};
  uint8_t* host[OMNI_MAX_CLASSES] = {};
  for (int k = 0; k < c.n_classes; ++k)
    if (labels_host[k] && (class_mask >> k & 1u)) {
      o.labels[k] = ws + p.lab[k];
      host[k] = labels_host[k];
    }
  if (!ctx->copy_st) OMNI_CU(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking), "copy stream");
  // every label band is downloaded on the copy stream as soon as it is stitched
  ctx->host_labels = host;
  r = omni_segment_slide(ctx, ws + p.in, H, W, dstride, scale_mask, class_mask, ws_, ws_bytes, &o, stream);
  ctx->host_labels = nullptr;
  if (r) {
    cudaStreamSynchronize(ctx->copy_st);
    return r;
  }
  OMNI_CU(cudaStreamSynchronize(st), "sync");
  unsigned herr = 0;
  OMNI_CU(cudaMemcpy(&herr, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
  if (herr) return fail(ctx, OMNI_ETIMEOUT, "a device-side wait gave up");
  return OMNI_OK;
}

}  // extern "C"

// ====================================================================== several slides per call
namespace {

// Workspace of a multi-slide call: every slide's tile stage (its own plan,
// laid out from prep_off[i]), the merged tile lists of every scale, then one
// network stage planned for the largest slide dimensions (its ring holds the
// widest slide's tile rows).
struct MultiPlan {
  int n = 0;
  Plan sp[OMNI_MAX_SLIDES];
  size_t prep_off[OMNI_MAX_SLIDES];
  size_t merged = 0;
  Plan net;
  size_t net_base = 0;     // ws + net_base + net.<region> addresses a network region
  size_t total = 0;
};

bool make_multi_plan(const omni_config& c, int n, const int32_t* H, const int32_t* W, MultiPlan& m) {
  if (n < 1 || n > OMNI_MAX_SLIDES) return false;
  m.n = n;
  size_t off = 0, ntile = 0;
  int Hm = 0, Wm = 0;
  for (int i = 0; i < n; ++i) {
    if (!make_plan(c, H[i], W[i], m.sp[i])) return false;
    m.prep_off[i] = off;
    off += align_up(m.sp[i].tile_end, 256);
    ntile += (size_t)m.sp[i].g.grid_off[c.n_scales];
    Hm = std::max(Hm, H[i]);
    Wm = std::max(Wm, W[i]);
  }
  m.merged = off;
  off = align_up(off + ntile * 3 * 4, 256);
  if (!make_plan(c, Hm, Wm, m.net)) return false;
  off = std::max(off, m.net.tile_end);
  m.net_base = off - m.net.tile_end;
  m.total = align_up(off + (m.net.net_end - m.net.tile_end), 256);
  return true;
}

// device clock (ns) at this point of the stream
__global__ void k_stamp(unsigned long long* out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  *out = t;
}

// merged list entry k = (slide, y, x) of the slide's tile k of one scale
__global__ void k_merge_tiles(const int32_t* __restrict__ src, int n, int slide, int32_t* __restrict__ dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  dst[3 * k] = slide;
  dst[3 * k + 1] = src[3 * k + 1];
  dst[3 * k + 2] = src[3 * k + 2];
}

}  // namespace

extern "C" {

omni_status omni_query_slides(const omni_config* cfg, int32_t n, const int32_t* H, const int32_t* W,
                              uint64_t* workspace_bytes) {
  if (!cfg || !H || !W || !workspace_bytes || !validate(*cfg).empty()) return OMNI_EINVAL;
  MultiPlan m;
  if (!make_multi_plan(*cfg, n, H, W, m)) return OMNI_EINVAL;
  *workspace_bytes = m.total;
  return OMNI_OK;
}

omni_status omni_segment_slides(omni_ctx* ctx, int32_t n, const uint8_t* const* rgb, const int32_t* H,
                                const int32_t* W, const int64_t* stride, uint32_t scale_mask,
                                uint32_t class_mask, void* ws_, uint64_t ws_bytes, const omni_outputs* out,
                                uint64_t* slide_ns, void* stream) {
  (void)cudaGetLastError();
  if (!ctx || !rgb || !H || !W || !stride || !out) return fail(ctx, OMNI_EINVAL, "null argument");
  if (!ctx->have_weights) return fail(ctx, OMNI_ESTATE, "omni_load_weights has not been called");
  if (n < 1 || n > OMNI_MAX_SLIDES) return fail(ctx, OMNI_EINVAL, "1..OMNI_MAX_SLIDES slides per call");
  const omni_config& c = ctx->cfg;
  for (int i = 0; i < n; ++i) {
    if (!rgb[i]) return fail(ctx, OMNI_EINVAL, "null slide " + std::to_string(i));
    if (stride[i] < (int64_t)W[i] * 3) return fail(ctx, OMNI_EINVAL, "row_stride < 3 W for slide " + std::to_string(i));
  }
  static thread_local MultiPlan mp;
  if (!make_multi_plan(c, n, H, W, mp)) return fail(ctx, OMNI_EINVAL, "bad slide size");
  omni_status r = check_ws(ctx, ws_, ws_bytes, mp.total);
  if (r) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  uint8_t* wsn = ws + mp.net_base;
  ctx->launches = 0;
  ctx->tiles_done = 0;
  ctx->band_ev_used = 0;
  // ---------------------------------------------------------------- every slide's tiling
  std::vector<Prep> pr(n);
  size_t nflags = 0;
  for (int i = 0; i < n; ++i) {
    r = run_prep(ctx, rgb[i], stride[i], mp.sp[i], ws + mp.prep_off[i], st, pr[i]);
    if (r) return r;
    nflags += (size_t)mp.sp[i].g.grid_off[c.n_scales];
  }
  if (ctx->h_flags_n < nflags) {
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    ctx->h_flags = nullptr;
    ctx->h_flags_n = 0;
    OMNI_CU(cudaMallocHost(&ctx->h_flags, nflags), "pinned tile flags");
    ctx->h_flags_n = nflags;
  }
  const int ncnt = 1 + c.n_scales;
  std::vector<size_t> foff(n);
  for (int i = 0, acc = 0; i < n; ++i) {
    const Plan& p = mp.sp[i];
    uint8_t* wp = ws + mp.prep_off[i];
    foff[i] = (size_t)acc;
    acc += p.g.grid_off[c.n_scales];
    OMNI_CU(cudaMemcpyAsync(ctx->h_counts + i * ncnt, wp + p.counts, ncnt * 4, cudaMemcpyDeviceToHost, st),
            "read tile counts");
    OMNI_CU(cudaMemcpyAsync(ctx->h_flags + foff[i], wp + p.flags, (size_t)p.g.grid_off[c.n_scales],
                            cudaMemcpyDeviceToHost, st),
            "read tile flags");
  }
  OMNI_CU(cudaStreamSynchronize(st), "sync after tiling");
  unsigned herr = 0;
  OMNI_CU(cudaMemcpy(&herr, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
  if (herr) return fail(ctx, OMNI_ETIMEOUT, "a device-side wait gave up in an earlier call");
  // per slide and scale: foreground tiles in grid rows 0..i, and the slide's
  // offset in the scale's merged list
  std::vector<std::vector<std::vector<int>>> row_end(n, std::vector<std::vector<int>>(c.n_scales));
  std::vector<std::array<int, OMNI_MAX_SCALES>> moff(n);
  std::array<int, OMNI_MAX_SCALES> N{}, soff{};
  for (int s = 0; s < c.n_scales; ++s) {
    for (int i = 0; i < n; ++i) {
      moff[i][s] = N[s];
      N[s] += ctx->h_counts[i * ncnt + 1 + s];
      const Plan& p = mp.sp[i];
      const uint8_t* fl = ctx->h_flags + foff[i] + p.g.grid_off[s];
      int acc = 0;
      row_end[i][s].resize(p.g.gh[s]);
      for (int y = 0; y < p.g.gh[s]; ++y) {
        for (int x = 0; x < p.g.gw[s]; ++x) acc += fl[(size_t)y * p.g.gw[s] + x] ? 1 : 0;
        row_end[i][s][y] = acc;
      }
    }
    if (s + 1 < c.n_scales) soff[s + 1] = soff[s] + N[s];
  }
  std::vector<uint64_t> key = {0x51u, (uint64_t)n, scale_mask, class_mask, reinterpret_cast<uint64_t>(ws_),
                               reinterpret_cast<uint64_t>(st)};
  for (int i = 0; i < n; ++i) {
    key.insert(key.end(), {reinterpret_cast<uint64_t>(rgb[i]), (uint64_t)H[i], (uint64_t)W[i], (uint64_t)stride[i]});
    for (int q = 0; q < ncnt; ++q) key.push_back((uint64_t)ctx->h_counts[i * ncnt + q]);
    for (int s = 0; s < c.n_scales; ++s)
      for (int v : row_end[i][s]) key.push_back((uint64_t)v);
    for (int k = 0; k < OMNI_MAX_CLASSES; ++k) {
      key.push_back(reinterpret_cast<uint64_t>(out[i].labels[k]));
      key.push_back(reinterpret_cast<uint64_t>(out[i].logits[k]));
    }
    for (int s = 0; s < OMNI_MAX_SCALES; ++s) {
      key.push_back(reinterpret_cast<uint64_t>(out[i].coverage[s]));
      key.push_back(reinterpret_cast<uint64_t>(out[i].argmax[s]));
    }
  }
  key.push_back(reinterpret_cast<uint64_t>(slide_ns));
  int last_scale = -1;
  for (int s = 0; s < c.n_scales; ++s) {
    int cls[OMNI_MAX_CLASSES];
    if ((scale_mask >> s & 1u) && classes_at(c, s, class_mask, cls) > 0) last_scale = s;
  }
  int32_t* merged = reinterpret_cast<int32_t*>(ws + mp.merged);
  // ---------------------------------------------------------------- network over the merged lists
  auto chain = [&](double& sb) -> omni_status {
    if (slide_ns) {
      k_stamp<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long*>(slide_ns));
      OMNI_CU(cudaGetLastError(), "slide stamp");
    }
    for (int s = 0; s < c.n_scales; ++s) {
      int cls[OMNI_MAX_CLASSES];
      const int ncls = classes_at(c, s, class_mask, cls);
      if (!(scale_mask >> s & 1u) || ncls == 0) continue;
      int32_t* ms = merged + 3 * (size_t)soff[s];
      CanvasTab cv{};
      std::vector<Bands> bands;
      for (int i = 0; i < n; ++i) {
        const Plan& p = mp.sp[i];
        const int n_is = ctx->h_counts[i * ncnt + 1 + s];
        cv.ptr[i] = pr[i].c[s];
        cv.stride[i] = pr[i].cs[s];
        cv.rows[i] = pr[i].ch[s];
        if (n_is > 0) {
          // the slide's list holds its scales in order: scale s starts after the earlier scales' tiles
          const int32_t* src = reinterpret_cast<const int32_t*>(ws + mp.prep_off[i] + p.tiles);
          int before = 0;
          for (int q = 0; q < s; ++q) before += ctx->h_counts[i * ncnt + 1 + q];
          k_merge_tiles<<<(n_is + 255) / 256, 256, 0, st>>>(src + 3 * (size_t)before, n_is, i, ms + 3 * (size_t)moff[i][s]);
          OMNI_CU(cudaGetLastError(), "merge tiles");
          ctx->launches++;
        }
        bands.push_back(make_bands(ctx, c, p, ws + mp.prep_off[i], wsn, mp.net, &out[i], H[i], W[i], s, cls, ncls,
                                   n_is, moff[i][s], row_end[i][s], sb));
      }
      const int cap = mp.net.cap[s];
      for (int start = 0; start < N[s]; start += c.max_batch) {
        const int nb = std::min(c.max_batch, N[s] - start);
        omni_status rr = run_batch(ctx, mp.net, wsn, s, cv, ms + 3 * (size_t)start, nb, start % cap, ncls, cls, st);
        if (rr) return rr;
        // stitch every band that became final in the slides this batch touched
        for (int i = 0; i < n; ++i) {
          const int lo = moff[i][s], n_is = ctx->h_counts[i * ncnt + 1 + s];
          if (n_is == 0 || lo >= start + nb || lo + n_is <= start) continue;
          rr = bands[i].advance(ctx, std::min(start + nb - lo, n_is), st);
          if (rr) return rr;
        }
      }
      for (int i = 0; i < n; ++i) {
        omni_status rr = bands[i].finish(ctx, st);
        if (rr) return rr;
        if (s == last_scale && slide_ns) {
          k_stamp<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long*>(slide_ns) + 1 + i);
          OMNI_CU(cudaGetLastError(), "slide stamp");
        }
      }
      ctx->tiles_done += N[s];
    }
    return OMNI_OK;
  };
  double stitch_bytes = 0;
  r = run_graphed(ctx, key, st, stitch_bytes, chain);
  if (r) return r;
  ctx->work[0] += (double)ctx->tiles_done * (double)mp.net.flops_per_tile;
  ctx->work[1] += stitch_bytes;
  return OMNI_OK;
}

omni_status omni_synth_slide(const int64_t* ell, int32_t n_ell, uint64_t seed, int32_t structures,
                             int32_t slide_w, int32_t y0, int32_t x0, int32_t h, int32_t w, uint8_t* out,
                             int64_t stride, void* stream) {
  if ((!ell && n_ell) || !out || n_ell < 0 || n_ell > kMaxEll || stride < (int64_t)w * 3) return OMNI_EINVAL;
  (void)cudaGetLastError();
  for (int k = 0; k < n_ell; ++k)
    if (ell[k * 6 + 2] <= 0 || ell[k * 6 + 3] <= 0) return OMNI_EINVAL;
  cudaError_t e = launch_synth(ell, n_ell, seed, structures != 0, slide_w, y0, x0, h, w, out, stride,
                               static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? OMNI_OK : OMNI_ECUDA;
}

}  // extern "C"

namespace {

// The E4M3 experiment of omni_conv_layer: activation scale s_x = max|x| / 448
// and weight scales s_w[o] = max_k |w[o][k]| / 448 (448 = the largest finite
// E4M3 value), so the quantised operands use the whole E4M3 range; the
// product of the two scales and g rides in the epilogue's per-channel scale.
omni_status conv_layer_e4m3(int32_t B, int32_t R, int32_t cin, int32_t cout, const void* x, int32_t x_cs,
                            int32_t x_co, const float* w_host, const float* g_host, const float* b_host,
                            void* y, int32_t y_cs, int32_t y_co, const int32_t* config, int32_t repeat,
                            float* ms_per_launch, cudaStream_t st) {
  if (x_cs != cin || x_co != 0 || cin % 128 || cout % 128 || cout > 512) return OMNI_EINVAL;
  if (!(R == 16 || R == 32 || R == 64 || (R >= 128 && R % 128 == 0))) return OMNI_EINVAL;
  TcConfig cfg{(long long)R * R % 256 == 0 ? 8 : 0, cout % 256 == 0 ? 256 : 128, 128, 0};
  if (config) {
    if (!((config[0] == 0 || config[0] == 8) && (config[1] == 128 || config[1] == 256) && config[2] == 128 &&
          config[3] == 0))
      return OMNI_EINVAL;
    cfg = TcConfig{config[0], config[1], config[2], 0};
  }
  const size_t K = (size_t)9 * cin;
  const long long n = (long long)B * R * R * cin;
  size_t off = 0;
  const size_t o_w = take(off, (size_t)cout * K), o_g = take(off, (size_t)cout * 4), o_b = take(off, (size_t)cout * 4),
               o_amax = take(off, 4), o_err = take(off, 4), o_x = take(off, (size_t)n);
  uint8_t* d = nullptr;
  if (cudaMalloc(&d, align_up(off, 256)) != cudaSuccess) return OMNI_ECUDA;
  omni_status rs = OMNI_OK;
  unsigned amax_bits = 0;
  cudaError_t e = cudaMemsetAsync(d + o_amax, 0, 4, st);      // max |x|
  if (e == cudaSuccess) e = cudaMemsetAsync(d + o_err, 0, 4, st);   // the kernels' status word
  if (e == cudaSuccess) e = launch_absmax_bf16(x, n, reinterpret_cast<unsigned*>(d + o_amax), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&amax_bits, d + o_amax, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float amax = 0.f;
  memcpy(&amax, &amax_bits, 4);
  const double s_x = amax > 0.f ? (double)amax / 448.0 : 1.0;
  if (e == cudaSuccess) e = launch_quant_e4m3(x, n, (float)(1.0 / s_x), d + o_x, st);
  // weight rows [cout][9 cin] (tap-major K, as the 16-bit paths) in E4M3
  std::vector<uint8_t> wq((size_t)cout * K);
  std::vector<float> gs(cout);
  for (int o = 0; o < cout; ++o) {
    float m = 0.f;
    for (size_t k = 0; k < K; ++k) m = std::max(m, std::fabs(w_host[(size_t)o * K + k]));
    const double s_w = m > 0.f ? (double)m / 448.0 : 1.0;
    for (int ci = 0; ci < cin; ++ci)
      for (int tap = 0; tap < 9; ++tap)
        wq[(size_t)o * K + (size_t)tap * cin + ci] = __nv_cvt_float_to_fp8(
            (float)(w_host[((size_t)o * cin + ci) * 9 + tap] / s_w), __NV_SATFINITE, __NV_E4M3);
    gs[o] = (float)(g_host[o] * s_x * s_w);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_w, wq.data(), wq.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_g, gs.data(), (size_t)cout * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_b, b_host, (size_t)cout * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    ConvArgs a{};
    a.B = B; a.R = R; a.cin = cin; a.cout = cout;
    a.x = d + o_x; a.x_cs = cin; a.x_co = 0;
    a.res_mode = RES_NONE;
    a.y = y; a.y_cs = y_cs; a.y_co = y_co;
    a.w.cin = cin; a.w.cout = cout;
    a.w.w_bf16 = reinterpret_cast<__nv_bfloat16*>(d + o_w);     // E4M3 bytes
    a.w.gamma = reinterpret_cast<float*>(d + o_g);
    a.w.beta = reinterpret_cast<float*>(d + o_b);
    a.err = reinterpret_cast<unsigned*>(d + o_err);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_per_launch) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    for (int i = 0; i < repeat && e == cudaSuccess; ++i) e = launch_conv_tc_e4m3(a, cfg, st);
    if (ms_per_launch) cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ms_per_launch) {
      float t = 0;
      if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
      *ms_per_launch = t / repeat;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, d + o_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && herr) rs = OMNI_ETIMEOUT;
  }
  if (e == cudaErrorInvalidValue) rs = OMNI_EINVAL;
  else if (e != cudaSuccess) rs = OMNI_ECUDA;
  cudaFree(d);
  return rs;
}

}  // namespace

extern "C" {

omni_status omni_conv_layer(int32_t precision, int32_t B, int32_t R, int32_t cin, int32_t cout,
                            const void* x, int32_t x_cs, int32_t x_co, const float* w_host,
                            const float* g_host, const float* b_host, const void* r, int32_t r_cs,
                            int32_t r_co, int32_t cr, const float* wp_host, void* y, int32_t y_cs,
                            int32_t y_co, const int32_t* config, int32_t repeat, float* ms_per_launch,
                            void* stream) {
  if (repeat < 1) return OMNI_EINVAL;
  if (precision == OMNI_E4M3) {
    if (!x || !y || !w_host || !g_host || !b_host || B <= 0 || R <= 0 || cin <= 0 || cout <= 0 || r)
      return OMNI_EINVAL;
    return conv_layer_e4m3(B, R, cin, cout, x, x_cs, x_co, w_host, g_host, b_host, y, y_cs, y_co, config,
                           repeat, ms_per_launch, static_cast<cudaStream_t>(stream));
  }
  if (!x || !y || !w_host || !g_host || !b_host || B <= 0 || R <= 0 || cin <= 0 || cout <= 0) return OMNI_EINVAL;
  if (cin % 8 || cout % 8 || (r && (cr <= 0 || cr % 8 || !wp_host))) return OMNI_EINVAL;
  if (precision != OMNI_FP32 && precision != OMNI_BF16 && precision != OMNI_FP16) return OMNI_EINVAL;
  const bool f16 = precision == OMNI_FP16;
  if (precision != OMNI_FP32 && !conv_tc_supported(R, cin, cout, r ? cr : 0)) return OMNI_EINVAL;
  TcConfig cfg{};
  if (precision != OMNI_FP32) {
    cfg = tc_default(R, cin, cout, r ? cr : 0);
    if (config) {
      TcConfig cands[16];
      const int n = tc_candidates(R, cin, cout, r ? cr : 0, cands, 16);
      bool found = false;
      // a candidate's kind, N tile and chunk with at most its pipeline stages
      for (int i = 0; i < n && !found; ++i)
        found = cands[i].kind == config[0] && cands[i].bn == config[1] && cands[i].ck == config[2] &&
                config[3] <= cands[i].stages && (cands[i].stages == 0 ? config[3] == 0 : config[3] >= 2);
      if (!found) return OMNI_EINVAL;
      cfg = TcConfig{config[0], config[1], config[2], config[3]};
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t n9 = (size_t)9 * cin * cout, np = r ? (size_t)cr * cout : 0;
  std::vector<float> w32(n9), wp32(np);
  std::vector<uint16_t> w16(n9), wp16(np);
  for (int o = 0; o < cout; ++o)
    for (int ci = 0; ci < cin; ++ci)
      for (int tap = 0; tap < 9; ++tap) {
        float v = w_host[((size_t)o * cin + ci) * 9 + tap];
        w32[((size_t)tap * cin + ci) * cout + o] = v;
        w16[(size_t)o * 9 * cin + (size_t)tap * cin + ci] = to_lp(v, f16);
      }
  for (int o = 0; o < cout && r; ++o)
    for (int ci = 0; ci < cr; ++ci) {
      float v = wp_host[(size_t)o * cr + ci];
      wp32[(size_t)ci * cout + o] = v;
      wp16[(size_t)o * cr + ci] = to_lp(v, f16);
    }
  size_t off = 0;
  size_t o32 = take(off, n9 * 4), o16 = take(off, n9 * 2), op32 = take(off, np * 4 + 4),
         op16 = take(off, np * 2 + 4), og = take(off, cout * 4), ob = take(off, cout * 4);
  std::vector<uint8_t> host(align_up(off, 256));
  memcpy(host.data() + o32, w32.data(), n9 * 4);
  memcpy(host.data() + o16, w16.data(), n9 * 2);
  if (np) {
    memcpy(host.data() + op32, wp32.data(), np * 4);
    memcpy(host.data() + op16, wp16.data(), np * 2);
  }
  memcpy(host.data() + og, g_host, cout * 4);
  memcpy(host.data() + ob, b_host, cout * 4);
  uint8_t* d = nullptr;
  unsigned* derr = nullptr;
  if (cudaMalloc(&d, host.size()) != cudaSuccess) return OMNI_ECUDA;
  if (cudaMalloc(&derr, sizeof(unsigned)) != cudaSuccess) { cudaFree(d); return OMNI_ECUDA; }
  omni_status rs = OMNI_OK;
  cudaError_t e = cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    ConvArgs a{};
    a.B = B; a.R = R; a.cin = cin; a.cout = cout;
    a.x = x; a.x_cs = x_cs; a.x_co = x_co;
    a.r = r; a.r_cs = r_cs; a.r_co = r_co; a.cr = r ? cr : 0;
    a.res_mode = r ? RES_TENSOR : RES_NONE;
    a.y = y; a.y_cs = y_cs; a.y_co = y_co;
    a.w.cin = cin; a.w.cout = cout; a.w.cproj = a.cr;
    a.w.w_f32 = reinterpret_cast<float*>(d + o32);
    a.w.w_bf16 = reinterpret_cast<__nv_bfloat16*>(d + o16);
    a.w.wp_f32 = reinterpret_cast<float*>(d + op32);
    a.w.wp_bf16 = reinterpret_cast<__nv_bfloat16*>(d + op16);
    a.w.gamma = reinterpret_cast<float*>(d + og);
    a.w.beta = reinterpret_cast<float*>(d + ob);
    a.err = derr;
    a.f16 = f16 ? 1 : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_per_launch) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    for (int i = 0; i < repeat && e == cudaSuccess; ++i)
      e = precision == OMNI_FP32 ? launch_conv_f32(a, st) : launch_conv_tc_cfg(a, cfg, st);
    if (ms_per_launch) cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ms_per_launch) {
      float t = 0;
      if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
      *ms_per_launch = t / repeat;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && herr) rs = OMNI_ETIMEOUT;
  }
  if (e != cudaSuccess) rs = OMNI_ECUDA;
  cudaFree(d);
  cudaFree(derr);
  return rs;
}

int32_t omni_conv_candidates(int32_t R, int32_t cin, int32_t cout, int32_t cr, int32_t* rows,
                             int32_t max_rows) {
  if (!rows || max_rows < 1 || R <= 0 || cin <= 0 || cout <= 0 || cr < 0) return 0;
  TcConfig cands[16];
  const int n = tc_candidates(R, cin, cout, cr, cands, 16);
  int k = 0;
  for (; k < n && k < max_rows; ++k) {
    rows[4 * k] = cands[k].kind;
    rows[4 * k + 1] = cands[k].bn;
    rows[4 * k + 2] = cands[k].ck;
    rows[4 * k + 3] = cands[k].stages;
  }
  return k;
}

omni_status omni_set_timing(omni_ctx* ctx, int32_t enabled) {
  if (!ctx) return OMNI_EINVAL;
  ctx->timing = enabled != 0;
  ctx->ev_used = 0;
  for (int k = 0; k < 4; ++k) ctx->work[k] = 0;
  return OMNI_OK;
}

omni_status omni_get_timing(omni_ctx* ctx, int32_t kind, double* ms, int64_t* launches, double* work) {
  if (!ctx || kind < 0 || kind > 3) return fail(ctx, OMNI_EINVAL, "bad timing kind");
  double tot = 0;
  int64_t n = 0;
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    if (ctx->evs[i].kind != kind) continue;
    float t = 0;
    cudaError_t e = cudaEventSynchronize(ctx->evs[i].b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ctx->evs[i].a, ctx->evs[i].b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event timing");
    tot += t;
    ++n;
  }
  if (ms) *ms = tot;
  if (launches) *launches = n;
  if (work) *work = ctx->work[kind];
  return OMNI_OK;
}

int64_t omni_last_launch_count(const omni_ctx* ctx) { return ctx ? ctx->launches : -1; }

omni_status omni_set_autotune(omni_ctx* ctx, int32_t enabled) {
  if (!ctx) return OMNI_EINVAL;
  ctx->autotune = enabled != 0;
  drop_graph(ctx);
  return OMNI_OK;
}

omni_status omni_set_e4m3(omni_ctx* ctx, int32_t enabled) {
  if (!ctx) return OMNI_EINVAL;
  if (enabled && ctx->cfg.precision != OMNI_BF16) return fail(ctx, OMNI_EINVAL, "the E4M3 experiment needs a BF16 context");
  ctx->e4m3 = enabled != 0;
  drop_graph(ctx);
  return OMNI_OK;
}

omni_status omni_set_conv_kind(omni_ctx* ctx, int32_t kind) {
  if (!ctx || kind < -1 || kind > 8) return OMNI_EINVAL;
  ctx->force_kind = kind;
  ctx->tuned.clear();          // forced choices are recorded there; the autotuner starts afresh
  drop_graph(ctx);
  return OMNI_OK;
}

omni_status omni_set_graphs(omni_ctx* ctx, int32_t enabled) {
  if (!ctx) return OMNI_EINVAL;
  ctx->graphs = enabled != 0;
  drop_graph(ctx);
  return OMNI_OK;
}

omni_status omni_set_fusion(omni_ctx* ctx, int32_t enabled) {
  if (!ctx) return OMNI_EINVAL;
  ctx->fuse = enabled != 0;
  drop_graph(ctx);
  return OMNI_OK;
}

int32_t omni_get_tuned(const omni_ctx* ctx, int32_t* rows, int32_t max_rows) {
  if (!ctx) return -1;
  int32_t n = 0;
  for (const auto& kv : ctx->tuned) {
    if (rows && n < max_rows) {
      int32_t* r = rows + 10 * n;
      for (int q = 0; q < 6; ++q) r[q] = kv.first[q];
      r[6] = kv.second.kind; r[7] = kv.second.bn; r[8] = kv.second.ck; r[9] = kv.second.stages;
    }
    ++n;
  }
  return n;
}

int64_t omni_get_launch_times(omni_ctx* ctx, int64_t max, double* ms, int32_t* kinds, int32_t* tags,
                              double* work) {
  if (!ctx) return -1;
  int64_t n = 0;
  for (size_t i = 0; i < ctx->ev_used && n < max; ++i, ++n) {
    float t = 0;
    if (cudaEventSynchronize(ctx->evs[i].b) != cudaSuccess ||
        cudaEventElapsedTime(&t, ctx->evs[i].a, ctx->evs[i].b) != cudaSuccess)
      return -1;
    if (ms) ms[n] = t;
    if (kinds) kinds[n] = ctx->evs[i].kind;
    if (tags) tags[n] = ctx->evs[i].tag;
    if (work) work[n] = ctx->evs[i].work;
  }
  return n;
}

}  // extern "C"

// ====================================================================== tiling without allocation
// omni_tile_slide_noalloc serves callers that may not allocate device memory
// while they run (see omniseg.h).  Its scratch is this file-scope array, which
// every GPU that loads the library holds until the process exits.  Host code
// must not pass the symbol itself to a kernel: on the host it names a stand-in
// object, not device memory.  The device address is looked up once per device
// with cudaGetSymbolAddress and cached.
namespace {

constexpr size_t kNoAllocScratch = 13u << 20;
static __device__ __align__(256) uint8_t g_tile_scratch[kNoAllocScratch];

std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};

// Device address of g_tile_scratch on the current device (set-up on first use).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tile_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Thumbnail grey straight from the caller's slide: one warp per 32x32 block of
// the padded 40x canvas, lane = column inside the block, the warp walking the
// block's 32 rows so each row read is 96 contiguous bytes; canvas pixels
// outside the slide take the 2x2-mean pad colour, so no padded copy of the
// slide is needed.
__global__ void k_thumb_direct(const uint8_t* __restrict__ rgb, long long stride, SlideGeom g,
                               uint8_t* __restrict__ grey) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= g.th * g.tw) return;
  const int ty = warp / g.tw, tx = warp % g.tw;
  int pad[3];
  const int h2 = g.H > 1 ? 1 : 0, w2 = g.W > 1 ? 1 : 0;
  for (int c = 0; c < 3; ++c) {
    int s = rgb[c] + rgb[w2 * 3 + c] + rgb[(long long)h2 * stride + c] + rgb[(long long)h2 * stride + w2 * 3 + c];
    pad[c] = (s + 2) >> 2;
  }
  const int x = tx * kThumb + lane - g.lead;
  const bool xin = x >= 0 && x < g.W;
  int sum[3] = {0, 0, 0};
  for (int q = 0; q < kThumb; ++q) {
    const int y = ty * kThumb + q - g.lead;
    if (xin && y >= 0 && y < g.H) {
      const uint8_t* p = rgb + (long long)y * stride + (long long)x * 3;
      sum[0] += p[0]; sum[1] += p[1]; sum[2] += p[2];
    } else {
      sum[0] += pad[0]; sum[1] += pad[1]; sum[2] += pad[2];
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < 3; ++c) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
  if (lane == 0) {
    const int R = (sum[0] + 512) >> 10, G = (sum[1] + 512) >> 10, B = (sum[2] + 512) >> 10;
    grey[warp] = (uint8_t)((77 * R + 150 * G + 29 * B + 128) >> 8);
  }
}

}  // namespace

extern "C" omni_status omni_tile_slide_noalloc(const omni_config* cfg, const uint8_t* rgb, int32_t H,
                                               int32_t W, int64_t stride, const omni_tile_list* out,
                                               void* stream) {
  if (!cfg || !rgb || !out || !out->tiles || !out->counts) return OMNI_EINVAL;
  if (!validate(*cfg).empty() || stride < (int64_t)W * 3) return OMNI_EINVAL;
  if (cfg->min_tissue_area > 0) return OMNI_EINVAL;     // the fixed scratch has no room for the area filter
  (void)cudaGetLastError();   // a launch error left by an earlier, unrelated call is not this call's
  Plan p;
  if (!make_plan(*cfg, H, W, p)) return OMNI_EINVAL;
  const SlideGeom& g = p.g;
  const size_t thumb = (size_t)g.th * g.tw;
  const size_t ntile = (size_t)g.grid_off[cfg->n_scales];
  if (thumb > OMNI_NOALLOC_MAX_THUMB_PX || ntile > OMNI_NOALLOC_MAX_TILES) {
    fprintf(stderr,
            "omni_tile_slide_noalloc: slide needs a %dx%d thumbnail and %zu tile cells; the static "
            "scratch holds %d thumbnail pixels and %d tile cells\n",
            g.th, g.tw, ntile, OMNI_NOALLOC_MAX_THUMB_PX, OMNI_NOALLOC_MAX_TILES);
    return OMNI_EINVAL;
  }
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return OMNI_ECUDA;
  size_t off = 0;
  uint8_t* sc = static_cast<uint8_t*>(base);
  uint8_t* grey = sc + take(off, OMNI_NOALLOC_MAX_THUMB_PX);
  uint8_t* blur = sc + take(off, OMNI_NOALLOC_MAX_THUMB_PX);
  uint8_t* mask = sc + take(off, OMNI_NOALLOC_MAX_THUMB_PX);
  int32_t* hist = reinterpret_cast<int32_t*>(sc + take(off, 256 * 4));
  int32_t* otsu = reinterpret_cast<int32_t*>(sc + take(off, 4));
  uint8_t* flags = sc + take(off, OMNI_NOALLOC_MAX_TILES);
  int32_t* slot = reinterpret_cast<int32_t*>(sc + take(off, (size_t)OMNI_NOALLOC_MAX_TILES * 4));
  if (off > kNoAllocScratch) return OMNI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)((thumb * 32 + 255) / 256);
  k_thumb_direct<<<blocks, 256, 0, st>>>(rgb, stride, g, grey);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_tissue_grey(grey, g, cfg->median_k, blur, hist, otsu, mask, st);
  if (e == cudaSuccess)
    e = launch_tiles(mask, g, cfg->tissue_filter, out->tiles, out->counts, out->flags ? out->flags : flags,
                     slot, st);
  if (e == cudaSuccess && out->tissue) e = cudaMemcpyAsync(out->tissue, mask, thumb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && out->otsu) e = cudaMemcpyAsync(out->otsu, otsu, 4, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? OMNI_OK : OMNI_ECUDA;
}

// ====================================================================== backward
namespace {

struct BwdPlan {
  Plan f;                      // forward workspace (first part of the buffer)
  size_t lg[OMNI_MAX_CLASSES], dl[OMNI_MAX_CLASSES], cov[OMNI_MAX_SCALES];
  size_t loss_partial, sums, cls_ids;
  size_t c1, a1, c2, pr, y0, dy0pre, dc2, da1, da1pre, dc1, dh0, dh0pre;
  size_t dtheta, wpart;
  size_t acc_wc, acc_bc, acc_wh, acc_bh, acc_w1, acc_g1, acc_b1, acc_w2, acc_g2, acc_b2, acc_wp;
  size_t total;
};

bool make_bwd_plan(const omni_config& c, int H, int W, BwdPlan& b) {
  if (!make_plan(c, H, W, b.f)) return false;
  size_t off = b.f.total;
  const int C0 = widths(c, 0), Cb = widths(c, c.levels - 1);
  for (int k = 0; k < c.n_classes; ++k) {
    const int f = c.factors[c.class_scale[k]];
    const size_t n = (size_t)((H + f - 1) / f) * ((W + f - 1) / f);
    b.lg[k] = take(off, n * 4);
    b.dl[k] = take(off, n * 4);
  }
  for (int s = 0; s < c.n_scales; ++s) {
    const int f = c.factors[s];
    b.cov[s] = take(off, (size_t)((H + f - 1) / f) * ((W + f - 1) / f) * 2);
  }
  b.loss_partial = take(off, (size_t)OMNI_MAX_CLASSES * loss_blocks() * 4 * 4);
  b.sums = take(off, (size_t)OMNI_MAX_CLASSES * 4 * 4);
  b.cls_ids = take(off, OMNI_MAX_CLASSES * 4);
  const size_t npx = (size_t)c.max_batch * c.patch * c.patch;
  const size_t fc = npx * C0 * 4;
  b.c1 = take(off, fc); b.a1 = take(off, fc); b.c2 = take(off, fc); b.pr = take(off, fc);
  b.y0 = take(off, fc); b.dy0pre = take(off, fc); b.dc2 = take(off, fc); b.da1 = take(off, fc);
  b.da1pre = take(off, fc); b.dc1 = take(off, fc);
  b.dh0 = take(off, npx * kHeadCh * 4); b.dh0pre = take(off, npx * kHeadCh * 4);
  b.dtheta = take(off, (size_t)c.max_batch * OMNI_MAX_CLASSES * head_bwd_blocks(c.patch) * kHeadParams * 4);
  b.wpart = take(off, (size_t)wgrad_chunks((long long)npx) * C0 * 27 * C0 * 4);
  const size_t zdim = Cb + c.n_classes + c.n_scales;
  b.acc_wc = take(off, (size_t)kHeadParams * zdim * 8);
  b.acc_bc = take(off, kHeadParams * 8);
  b.acc_wh = take(off, (size_t)kHeadCh * C0 * 8);
  b.acc_bh = take(off, kHeadCh * 8);
  b.acc_w1 = take(off, (size_t)C0 * 27 * C0 * 8);
  b.acc_g1 = take(off, C0 * 8);
  b.acc_b1 = take(off, C0 * 8);
  b.acc_w2 = take(off, (size_t)C0 * 9 * C0 * 8);
  b.acc_g2 = take(off, C0 * 8);
  b.acc_b2 = take(off, C0 * 8);
  b.acc_wp = take(off, (size_t)C0 * 3 * C0 * 8);
  b.total = align_up(off, 256);
  return true;
}

// [o][tap][c] (accumulation order, compensated (sum, carry) pairs) ->
// [o][c][tap] (blob order), FP32
__global__ void k_w_to_blob(const float2* __restrict__ acc, int O, int cin, int taps, float* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)O * cin * taps;
  if (i >= n) return;
  const int o = (int)(i / ((long long)cin * taps));
  const int rem = (int)(i % ((long long)cin * taps));
  const int c = rem / taps, t = rem % taps;
  const float2 a = acc[(long long)o * cin * taps + (long long)t * cin + c];
  out[i] = a.x - a.y;
}

}  // namespace

extern "C" uint64_t omni_backward_workspace(const omni_config* cfg, int32_t H, int32_t W) {
  if (!cfg || !validate(*cfg).empty()) return 0;
  BwdPlan b;
  if (!make_bwd_plan(*cfg, H, W, b)) return 0;
  return b.total;
}

extern "C" omni_status omni_backward(omni_ctx* ctx, const uint8_t* rgb, int32_t H, int32_t W, int64_t stride,
                                     const uint8_t* const* gt_dev, void* ws_, uint64_t ws_bytes, float* loss_dev,
                                     const omni_grads* grads, void* stream) {
  if (!ctx || !rgb || !gt_dev || !loss_dev || !grads) return fail(ctx, OMNI_EINVAL, "null argument");
  if (!ctx->have_weights) return fail(ctx, OMNI_ESTATE, "omni_load_weights has not been called");
  const omni_config& c = ctx->cfg;
  if (c.precision != OMNI_FP32) return fail(ctx, OMNI_EINVAL, "omni_backward needs an OMNI_FP32 context");
  if (c.stitch_window != OMNI_WINDOW_FLAT)
    return fail(ctx, OMNI_EINVAL, "omni_backward differentiates the flat overlap average only");
  for (int k = 0; k < c.n_classes; ++k)
    if (!gt_dev[k]) return fail(ctx, OMNI_EINVAL, "missing ground-truth mask for class " + std::to_string(k));
  BwdPlan bp;
  if (!make_bwd_plan(c, H, W, bp)) return fail(ctx, OMNI_EINVAL, "bad slide size");
  omni_status r = check_ws(ctx, ws_, ws_bytes, bp.total);
  if (r) return r;
  if (c.max_batch > 64) return fail(ctx, OMNI_EINVAL, "omni_backward supports max_batch <= 64");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  const Plan& p = bp.f;
  const int L = c.levels, C0 = widths(c, 0), Cb = widths(c, L - 1), P = c.patch;
  const long long PP = (long long)P * P;
  auto F = [&](size_t o) { return reinterpret_cast<float*>(ws + o); };
  auto D = [&](size_t o) { return reinterpret_cast<float2*>(ws + o); };   // compensated accumulators

  // ---------------------------------------------------------------- pass 1: forward
  omni_outputs fo{};
  for (int k = 0; k < c.n_classes; ++k) fo.logits[k] = F(bp.lg[k]);
  for (int s = 0; s < c.n_scales; ++s) fo.coverage[s] = reinterpret_cast<uint16_t*>(ws + bp.cov[s]);
  const uint32_t all_s = (1u << c.n_scales) - 1, all_c = (1u << c.n_classes) - 1;
  r = omni_segment_slide(ctx, rgb, H, W, stride, all_s, all_c, ws_, ws_bytes, &fo, stream);
  if (r) return r;

  // ---------------------------------------------------------------- loss and dloss/dL
  NPix npix{};
  for (int k = 0; k < c.n_classes; ++k) {
    const int f = c.factors[c.class_scale[k]];
    npix.n[k] = (long long)((H + f - 1) / f) * ((W + f - 1) / f);
    OMNI_CU(launch_loss_partial(F(bp.lg[k]), gt_dev[k], npix.n[k], F(bp.loss_partial) + (size_t)k * loss_blocks() * 4, st),
            "loss partial");
  }
  OMNI_CU(launch_loss_final(F(bp.loss_partial), c.n_classes, npix, F(bp.sums), loss_dev, st), "loss");
  for (int k = 0; k < c.n_classes; ++k)
    OMNI_CU(launch_loss_grad(F(bp.lg[k]), gt_dev[k], npix.n[k], F(bp.sums) + 4 * k, (float)npix.n[k],
                             c.n_classes, F(bp.dl[k]), st),
            "loss grad");
  OMNI_CU(cudaMemsetAsync(ws + bp.acc_wc, 0, bp.total - bp.acc_wc, st), "clear accumulators");

  // ---------------------------------------------------------------- pass 2: recompute + backward per batch
  Prep pr;
  {
    // canvases of every scale (integer stages, identical to pass 1)
    r = run_prep(ctx, rgb, stride, p, ws, st, pr);
    if (r) return r;
  }
  const int32_t* tiles = reinterpret_cast<const int32_t*>(ws + p.tiles);
  int32_t* cls_dev = reinterpret_cast<int32_t*>(ws + bp.cls_ids);
  int toff = 0;
  for (int s = 0; s < c.n_scales; ++s) {
    const int n_s = ctx->h_counts[1 + s];
    int cls[OMNI_MAX_CLASSES], ncls = 0;
    for (int k = 0; k < c.n_classes; ++k)
      if (c.class_scale[k] == s) cls[ncls++] = k;
    if (ncls == 0) { toff += n_s; continue; }
    const int f = c.factors[s];
    for (int start = 0; start < n_s; start += c.max_batch) {
      const int nb = std::min(c.max_batch, n_s - start);
      const int32_t* t3 = tiles + 3 * (toff + start);
      const long long npx = (long long)nb * PP;
      r = run_batch(ctx, p, ws, s, one_canvas(pr, s), t3, nb, start, ncls, cls, st, true);
      if (r) return r;
      void* cat0 = ws + p.cat[0];
      ConvArgs a{};
      a.B = nb; a.R = P; a.raw = 1; a.err = ctx->d_err;
      a.cin = 3 * C0; a.cout = C0; a.x = cat0; a.x_cs = 3 * C0; a.y = F(bp.c1); a.y_cs = C0; a.w = ctx->dec1[0];
      OMNI_CU(launch_conv_f32(a, st), "recompute conv1");
      OMNI_CU(launch_affine_relu(F(bp.c1), ctx->dec1[0].gamma, ctx->dec1[0].beta, C0, npx, F(bp.a1), st), "a1");
      ConvArgs b2{};
      b2.B = nb; b2.R = P; b2.raw = 1; b2.err = ctx->d_err;
      b2.cin = C0; b2.cout = C0; b2.x = F(bp.a1); b2.x_cs = C0; b2.y = F(bp.c2); b2.y_cs = C0;
      b2.res_mode = RES_TENSOR; b2.r = cat0; b2.r_cs = 3 * C0; b2.cr = 3 * C0; b2.y2 = F(bp.pr); b2.y2_cs = C0;
      b2.w = ctx->dec2[0];
      OMNI_CU(launch_conv_f32(b2, st), "recompute conv2");
      BwdHeadArgs h{};
      h.B = nb; h.P = P; h.n_cls = ncls;
      h.theta = F(p.theta);
      h.wh = ctx->wh; h.bh = ctx->bh; h.g2 = ctx->dec2[0].gamma; h.b2 = ctx->dec2[0].beta;
      h.tiles3 = t3;
      h.oy0 = c.pad_lead / f; h.ox0 = c.pad_lead / f; h.oh = (H + f - 1) / f; h.ow = (W + f - 1) / f;
      h.cov = reinterpret_cast<const uint16_t*>(ws + bp.cov[s]);
      h.c2 = F(bp.c2); h.pr = F(bp.pr); h.dh0 = F(bp.dh0); h.dtheta_partial = F(bp.dtheta);
      h.y0 = F(bp.y0); h.dh0_pre = F(bp.dh0pre); h.dy0_pre = F(bp.dy0pre); h.dc2 = F(bp.dc2);
      for (int ci = 0; ci < ncls; ++ci) {
        h.ci = ci;
        h.dL = F(bp.dl[cls[ci]]);
        OMNI_CU(launch_head_bwd(h, C0, st), "head backward");
      }
      OMNI_CU(launch_prehead_bwd(h, C0, npx, st), "pre-head backward");
      float* wpart = F(bp.wpart);
      OMNI_CU(launch_wgrad(F(bp.dh0pre), kHeadCh, F(bp.y0), C0, C0, 1, P, npx, wpart, D(bp.acc_wh), st), "dWh");
      OMNI_CU(launch_colsum(F(bp.dh0pre), nullptr, kHeadCh, npx, wpart, D(bp.acc_bh), st), "dbh");
      OMNI_CU(launch_colsum(F(bp.dy0pre), nullptr, C0, npx, wpart, D(bp.acc_b2), st), "db2");
      OMNI_CU(launch_colsum(F(bp.dy0pre), F(bp.c2), C0, npx, wpart, D(bp.acc_g2), st), "dg2");
      OMNI_CU(launch_wgrad(F(bp.dy0pre), C0, static_cast<const float*>(cat0), 3 * C0, 3 * C0, 1, P, npx, wpart,
                           D(bp.acc_wp), st), "dWp");
      OMNI_CU(launch_wgrad(F(bp.dc2), C0, F(bp.a1), C0, C0, 9, P, npx, wpart, D(bp.acc_w2), st), "dW2");
      ConvArgs dg{};
      dg.B = nb; dg.R = P; dg.raw = 1; dg.err = ctx->d_err;
      dg.cin = C0; dg.cout = C0; dg.x = F(bp.dc2); dg.x_cs = C0; dg.y = F(bp.da1); dg.y_cs = C0; dg.w = ctx->dec2t0;
      OMNI_CU(launch_conv_f32(dg, st), "da1");
      OMNI_CU(launch_relu_bwd(F(bp.da1), F(bp.c1), ctx->dec1[0].gamma, ctx->dec1[0].beta, C0, npx, F(bp.da1pre),
                              F(bp.dc1), st), "relu backward");
      OMNI_CU(launch_colsum(F(bp.da1pre), nullptr, C0, npx, wpart, D(bp.acc_b1), st), "db1");
      OMNI_CU(launch_colsum(F(bp.da1pre), F(bp.c1), C0, npx, wpart, D(bp.acc_g1), st), "dg1");
      OMNI_CU(launch_wgrad(F(bp.dc1), C0, static_cast<const float*>(cat0), 3 * C0, 3 * C0, 9, P, npx, wpart,
                           D(bp.acc_w1), st), "dW1");
      OMNI_CU(cudaMemcpyAsync(cls_dev, cls, ncls * sizeof(int32_t), cudaMemcpyHostToDevice, st), "class ids");
      OMNI_CU(launch_ctrl_bwd(F(bp.dtheta), head_bwd_blocks(P), nb, ncls, cls_dev, c.n_classes, c.n_scales, s,
                              F(p.gap), Cb, D(bp.acc_wc), D(bp.acc_bc), st), "controller backward");
      // the class-id upload reads host memory that changes next batch
      OMNI_CU(cudaStreamSynchronize(st), "batch sync");
    }
    toff += n_s;
  }

  // ---------------------------------------------------------------- FP32 outputs in blob layouts
  const long long zdim = Cb + c.n_classes + c.n_scales;
  auto out = [&](float* dst, size_t acc, long long n) -> cudaError_t {
    return dst ? launch_to_f32(D(acc), n, dst, st) : cudaSuccess;
  };
  OMNI_CU(out(grads->ctrl_w, bp.acc_wc, kHeadParams * zdim), "ctrl_w");
  OMNI_CU(out(grads->ctrl_b, bp.acc_bc, kHeadParams), "ctrl_b");
  OMNI_CU(out(grads->head_w, bp.acc_wh, (long long)kHeadCh * C0), "head_w");
  OMNI_CU(out(grads->head_b, bp.acc_bh, kHeadCh), "head_b");
  OMNI_CU(out(grads->dec0_g1, bp.acc_g1, C0), "g1");
  OMNI_CU(out(grads->dec0_b1, bp.acc_b1, C0), "b1");
  OMNI_CU(out(grads->dec0_g2, bp.acc_g2, C0), "g2");
  OMNI_CU(out(grads->dec0_b2, bp.acc_b2, C0), "b2");
  OMNI_CU(out(grads->dec0_wp, bp.acc_wp, (long long)C0 * 3 * C0), "wp");
  if (grads->dec0_w1) {
    const long long n = (long long)C0 * 3 * C0 * 9;
    k_w_to_blob<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D(bp.acc_w1), C0, 3 * C0, 9, grads->dec0_w1);
  }
  if (grads->dec0_w2) {
    const long long n = (long long)C0 * C0 * 9;
    k_w_to_blob<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D(bp.acc_w2), C0, C0, 9, grads->dec0_w2);
  }
  OMNI_CU(cudaGetLastError(), "gradient outputs");
  return OMNI_OK;
}
