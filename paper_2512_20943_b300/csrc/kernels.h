// Host-side launchers of the AirGS kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "airgs_internal.cuh"

#define AIRGS_MAX_VIEWS_DEV 256

namespace airgs {

// Process-wide count of kernel launches issued by the library.
void count_launches(int n);

cudaError_t launch_decode_apply(cudaStream_t st, int64_t n, const uint16_t* map, int64_t plane, const float* lo,
                                const float* hi, int quat_add, const float* base_means, const float* base_quats,
                                float* out_means, float* out_quats);

// Tile lists: kCullNone lists a Gaussian in every tile of its 3-sigma rectangle
// (the definition's lists), kCullBands only in the tiles where it can reach
// alpha_min (exact row bands of its ellipse), kCullBox in the tiles of the
// rectangle that the bounding box of that region meets (cheaper to compute,
// fewer tiles dropped).  Images, T, blend weights and gradients are the same.
constexpr int kCullNone = 0, kCullBands = 1, kCullBox = 2;

cudaError_t launch_project(cudaStream_t st, int64_t n, int sh_degree, const float* means, const float* log_scales,
                           const float* quats, const float* opacity_logit, const float* sh, const CamDev* cams,
                           int n_views, const RasterParams& rp, ProjRec* proj, uint32_t* depth_keys,
                           uint32_t* tiles_touched, uint32_t* tile_counts, int cull);

// Per-tile ordering (order.cu).
constexpr int kTileSortSmall = 2048;  // entries sorted by one 256-thread CTA
constexpr int kTileSortBig = 16384;   // entries sorted by one 1024-thread CTA
cudaError_t launch_tile_offsets(cudaStream_t st, const uint32_t* counts, int64_t n_tiles, uint64_t* chunk_sums,
                                uint2* ranges, uint32_t* cursor, uint32_t* big_list, uint32_t* info);
size_t tile_offsets_chunks(int64_t n_tiles);
cudaError_t launch_scatter(cudaStream_t st, int64_t total, int64_t n, const ProjRec* proj, const CamDev* cams,
                           const uint32_t* depth_keys, uint32_t* cursor, uint2* pairs);
// n_big: the number of long lists, or with n_big_dev (their count on the
// device) an upper bound on it.
cudaError_t launch_sort_tiles(cudaStream_t st, int64_t n_tiles, const uint2* ranges, const uint32_t* big_list,
                              int64_t n_big, const uint2* pairs, uint32_t* vals, const uint32_t* n_big_dev);

// keys: radix keys per thread (6, 8 or 12; 0 = the default for the segment
// count); the scratch size and the sort must be given the same value.
size_t radix_scratch_bytes(int64_t seg_len, int n_seg, int num_sms, int keys = 0);
cudaError_t radix_sort_pairs(cudaStream_t st, int num_sms, uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                             uint32_t* vals_b, int64_t seg_len, int n_seg, int key_bits, bool identity_vals,
                             uint32_t* scratch, bool* result_in_b, int keys = 0);

// One pass: the digit of bits [shift, min(shift + 8, key_bits)).
cudaError_t radix_sort_pass(cudaStream_t st, int num_sms, const uint32_t* keys_in, const uint32_t* vals_in,
                            uint32_t* keys_out, uint32_t* vals_out, int64_t n, int shift, int key_bits,
                            uint32_t* counts);

cudaError_t launch_count_gather(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                                const uint32_t* tiles_touched, uint32_t* counts_sorted, uint64_t* chunk_sums,
                                int64_t* n_chunks);
// Exclusive scan in place of n_chunks sums (and of a second array of the same
// length when sums2 is given, in the same launch); totals -> total_out(2).
cudaError_t launch_scan_spans(cudaStream_t st, uint64_t* sums, int64_t n_chunks, uint64_t* total_out,
                              uint64_t* sums2 = nullptr, uint64_t* total_out2 = nullptr);
size_t emit_piece_words(int64_t total, int64_t n_inst);
int64_t emit_chunks(int64_t total);  // depth-order chunks of the count/scan/emit kernels
cudaError_t launch_emit(cudaStream_t st, int64_t total, int64_t n, const uint32_t* order,
                        const uint32_t* counts_sorted, const uint64_t* chunk_offsets, int64_t n_inst,
                        uint32_t* piece_off, const ProjRec* proj, const CamDev* cams, float alpha_min,
                        int64_t n_tiles, int cull, int run, uint32_t* keys, uint32_t* vals);
cudaError_t launch_tile_ranges(cudaStream_t st, int64_t n_inst, const uint32_t* keys, uint2* ranges);

// Usage-frequency pruning (prune.cu).
cudaError_t launch_prune_mask(cudaStream_t st, int num_sms, int64_t n, int64_t n_prune, const float* w,
                              uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                              uint32_t* scratch, uint8_t* keep);
cudaError_t launch_prune_delta(cudaStream_t st, int64_t n, int channels, const float* D_t, float* D_sent,
                               const uint8_t* keep, float* d_out, unsigned long long* nonzero);
cudaError_t launch_apply_delta(cudaStream_t st, int64_t n, const float* delta, int quat_add, const float* base_means,
                               const float* base_quats, float* out_means, float* out_quats);
cudaError_t launch_densify_select(cudaStream_t st, int64_t n, const float* g, const uint32_t* views, float threshold,
                                  uint8_t* mask);
cudaError_t launch_sq_err(cudaStream_t st, const float* a, const float* b, const int64_t* view_off, int n_views,
                          double* out);

// Clone / split / discard of keyframe densification (densify.cu): scratch cls
// [n] bytes, tile_counts [densify_tiles(n)], totals [4].
int64_t densify_tiles(int64_t n);
cudaError_t launch_densify_apply(cudaStream_t st, int64_t n, int sh_degree, const float* means,
                                 const float* log_scales, const float* quats, const float* opacity_logit,
                                 const float* sh, const uint8_t* select, const float* z, float ls_thr, float ls_div,
                                 float lo_thr, uint8_t* cls, uint3* tile_counts, uint32_t* totals, float* o_means,
                                 float* o_log_scales, float* o_quats, float* o_opacity_logit, float* o_sh,
                                 uint32_t* o_parent, int64_t* n_out);

// L_3DGS = (1 - lambda) L1 + lambda (1 - SSIM) and its image gradient (ssim.cu):
// one CTA per 32x32 output tile of each (view, channel) plane; d_tile_base
// [n_planes + 1] the planes' first tiles (ssim_tiles per plane), n_tiles their
// total.  sums: 5 doubles (zeroed; [2..4] receive L, L1, SSIM).
int64_t ssim_tiles(int w, int h);
cudaError_t launch_ssim_loss(cudaStream_t st, const int64_t* d_off, const int* d_w, const int* d_h,
                             const int64_t* d_tile_base, int n_planes, int64_t total, int64_t n_tiles, const float* x,
                             const float* y, float lambda, double* sums, float* grad);

// Half-tile blend lists (cull_lists.cu).
size_t half_list_chunks(int64_t n_inst);
cudaError_t launch_half_lists(cudaStream_t st, const uint32_t* keys, const uint32_t* ids, uint2* ranges,
                              const CamDev* cams, int n_views, const ProjRec* proj, int64_t n, int64_t n_inst,
                              float alpha_min, int64_t n_tiles, uint8_t* flags, uint64_t* sums, uint2* hl,
                              uint2* hranges);
// Queue order of the blend kernels' 2 n_tiles half-tile items (work index
// 2 tile + half): groups of views_per_group consecutive views in view order,
// the last group taking the remaining views (at least last_views), within a
// group decreasing half-list length in bins of a quarter octave.  scratch:
// item_order_words words; order: 2 n_tiles words.
constexpr int kOrderBins = 64;
size_t item_order_words(int n_views);
cudaError_t launch_item_order(cudaStream_t st, int num_sms, const uint2* hranges, const CamDev* cams, int n_views,
                              int views_per_group, int last_views, int64_t n_tiles, uint32_t* scratch,
                              uint32_t* order);

struct BlendArgs {
  const ProjRec* proj;  // [V][N]
  int64_t n;
  const uint32_t* ids;  // sorted instance values (Gaussian ids)
  const uint2* ranges;  // [tiles] (start, end)
  const CamDev* cams;
  int n_views;
  int64_t n_tiles;
  RasterParams rp;
  int* work_counter;
  unsigned long long* pair_counter;
  unsigned long long* pair_total;  // nullable: cumulative counter of the context
  unsigned long long* exec_total;  // nullable: cumulative lane evaluations actually issued (32 per block)
  const uint2* hl;                 // nullable: half-tile lists of (Gaussian id, full-list position | block mask)
  uint2* hl_mut;                   // the same lists, written by the compacting forward (block masks)
  const uint2* hranges;            // [2][tiles] ranges into hl (top halves, then bottom halves)
  const uint32_t* work_order;      // nullable: the queue's work indices in the order to hand them out
};

struct FwdOut {
  float* rgb;        // planar per view
  float* T;          // nullable
  int32_t* ncontrib; // state copy (required)
  int32_t* ncontrib_user;  // nullable
  float* imp_w;      // nullable
  uint32_t* imp_cnt; // nullable
};

struct BwdIn {
  const float* rgb;     // final colour of the forward (C + T bg)
  const float* dL;      // dL/drgb (nullable when l1)
  const float* target;  // L1 target (nullable)
  float inv_norm;       // 1 / (3 sum H W)
  float* loss;          // L1 accumulator (nullable)
  const int32_t* ncontrib;
  GradRec* grad;        // [V][N]
  float* imp_w;         // nullable: usage frequency requested (the replay fills the records' weight
  uint32_t* imp_cnt;    // and count slots; the projection adjoint adds them here)
};

// Kernel shapes the autotuner searches: compiled instantiations of the blend
// forward and backward (staged list entries per batch, warps per SM: the
// register bound), keys per thread of the instances' radix sort and the
// emission's instances per thread.  A shape index packs (forward f, backward
// b, sort k, emission e) as f + kFwdShapes (b + kBwdShapes (k + kSortShapes e));
// shape 0 (every part 0) is the default.
constexpr int kFwdShapes = 5;   // forward (batch, warps): (32, 28) (16, 28) (64, 28) (32, 32) (32, 24)
constexpr int kBwdShapes = 5;   // backward (batch, warps): (32, 32) (16, 32) (64, 32) (32, 28) (32, 24)
constexpr int kSortShapes = 3;  // instance sort keys per thread: 8, 6, 12
constexpr int kEmitShapes = 3;  // emission instances per thread and piece: 8, 4, 16
constexpr int kShapes = kFwdShapes * kBwdShapes * kSortShapes * kEmitShapes;
struct ShapeParts {
  int fwd, bwd, sort, emit;
};
inline ShapeParts shape_parts(int shape) {
  if (shape < 0 || shape >= kShapes) shape = 0;
  return ShapeParts{shape % kFwdShapes, (shape / kFwdShapes) % kBwdShapes,
                    (shape / (kFwdShapes * kBwdShapes)) % kSortShapes, shape / (kFwdShapes * kBwdShapes * kSortShapes)};
}
inline int shape_index(int fwd, int bwd, int sort, int emit) {
  return fwd + kFwdShapes * (bwd + kBwdShapes * (sort + kSortShapes * emit));
}
inline int sort_keys_of(int sort_shape) { return sort_shape == 1 ? 6 : sort_shape == 2 ? 12 : 8; }
inline int emit_run_of(int emit_shape) { return emit_shape == 1 ? 4 : emit_shape == 2 ? 16 : 8; }
const char* shape_name(int shape);
cudaError_t launch_blend_fwd(cudaStream_t st, int fwd_shape, int num_sms, const BlendArgs& a, const FwdOut& o);
cudaError_t launch_blend_bwd(cudaStream_t st, int bwd_shape, int num_sms, const BlendArgs& a, const BwdIn& in);

cudaError_t launch_project_bwd(cudaStream_t st, int64_t n, int sh_degree, const float* means,
                               const float* log_scales, const float* quats, const float* opacity_logit,
                               const float* sh, const CamDev* cams, int n_views, const ProjRec* proj,
                               const GradRec* grad, float* g_means, float* g_log_scales, float* g_quats,
                               float* g_opacity, float* g_sh, float* dens_grad, uint32_t* dens_views, float* imp_w,
                               uint32_t* imp_cnt);

cudaError_t measure_fp32_peak(cudaStream_t st, int num_sms, float* scratch, double* tflops);
size_t fp32_probe_words(int num_sms);
cudaError_t measure_smem_peak(cudaStream_t st, int num_sms, float* scratch, double* tbs);
size_t smem_probe_words(int num_sms);

}  // namespace airgs
