// fmb_api.cu -- the C ABI of include/fmb.h: host-side validation, launch planning
// and the enqueueing of the prologue, forward, backward and reduction kernels.
// No device memory is allocated here; scratch lives in the caller's workspace:
//
//   [0, 256)            status word (int) at 0, forward work counter at 64,
//                       backward work counter at 128
//   [256, 256 + 64 R)   R per-(view, Gaussian) records, R = sum over views of K
//   [.., ..)            backward partials (deterministic mode only)
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <exception>
#include <mutex>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "fmb_internal.cuh"

namespace fmb {
int forward_rays_per_cta(int rpt);
}

// The Python binding mirrors these layouts field by field (ctypes structures).
static_assert(sizeof(fmb_params) == 68 && offsetof(fmb_params, bwd_gblocks) == 64, "fmb_params layout");
static_assert(sizeof(fmb_view) == 64 && offsetof(fmb_view, pix_offset) == 40, "fmb_view layout");

namespace {

thread_local std::string g_err;

constexpr size_t kHeaderBytes = 256;
constexpr size_t kFwdCounterOffset = 64;
constexpr size_t kBwdCounterOffset = 128;
constexpr int kDefaultRpt = 2;
constexpr int kMaxGaussPerCta = 256;
constexpr long long kMaxK = 1 << 22;
constexpr int kMaxKAlphaCompositing = 256;
constexpr long long kMaxGaussians = 0x7fffffffll;  // all objects together (32-bit Gaussian offsets)
constexpr long long kMaxRecords = 1ll << 28;       // sum over views of K (32-bit record offsets, 16 GB)

fmb_status fail(fmb_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Plane entries of a view: its ray batch, or the whole image.
long long view_entries(const fmb_view& v) {
  return v.rays != nullptr ? static_cast<long long>(v.n_rays) : static_cast<long long>(v.W) * v.H;
}

struct BwdBlocking {
  int n_gb, GB, S;
};

// Fraction of a CTA's thread lanes that carry a real (ray, Gaussian) pair when K
// Gaussians are split into n blocks for T threads.
static double bwd_lane_fill(int K, int T, int n) {
  const int GB = (K + n - 1) / n;
  const int gb2 = (GB + 1) / 2;
  const int S = std::max(1, T / gb2);
  return (static_cast<double>(gb2) * S / T) * (static_cast<double>(K) / (n * 2.0 * gb2));
}

// Backward blocking of K Gaussians for T threads: each thread owns two Gaussians
// (one per packed lane), so a CTA covers GB <= min(2T, 256) Gaussians with
// ceil(GB/2) threads per ray subgroup and S = T / ceil(GB/2) subgroups.  The block
// count is the fewest that fit, or up to three more where that fills the threads
// better: the modelled cost per ray is K / fill (pair work) plus 5 per block (the
// per-ray records each block builds), e.g. K = 200 at T = 160 runs as two blocks of
// 100 (3 subgroups of 50 threads) instead of one of 200 (one subgroup of 100).
// min_blocks > 0 (the bwd_gblocks hint) raises the count to at least that many,
// for batches too small to fill the GPU with one block per ray tile.  even_blocks
// (the stored-intermediate adjoint, which reads a thread's two Gaussians' stored
// values with one 8-byte load) rounds the block size up to an even count, so that
// every block starts at an even Gaussian index.
BwdBlocking bwd_blocking(int K, int T, int min_blocks = 0, bool even_blocks = false) {
  const int gbmax = std::min(2 * T, kMaxGaussPerCta);
  const int n_min = (K + gbmax - 1) / gbmax;
  int best_n = n_min;
  double best_cost = 0.0;
  for (int n = n_min; n <= std::min(K, n_min + 3); ++n) {
    const double cost = K / bwd_lane_fill(K, T, n) + 5.0 * n;
    if (n == n_min || cost < best_cost - 1e-9) {
      best_cost = cost;
      best_n = n;
    }
  }
  BwdBlocking b;
  b.n_gb = best_n;
  b.GB = (K + b.n_gb - 1) / b.n_gb;
  if (min_blocks > best_n) {
    // blocks of ceil(K / n) Gaussians, none of them empty
    b.GB = (K + std::min(min_blocks, K) - 1) / std::min(min_blocks, K);
    b.n_gb = (K + b.GB - 1) / b.GB;
  }
  if (even_blocks && b.n_gb > 1 && (b.GB & 1)) {
    b.GB += 1;  // at most min(2T, 256) still: that bound is even
    b.n_gb = (K + b.GB - 1) / b.GB;
  }
  b.S = std::max(1, T / ((b.GB + 1) / 2));
  return b;
}

// Threads per backward CTA: the candidate with the lowest modelled cost over the
// batch (each view's rays x (K / lane fill + 5 per Gaussian block), as in
// bwd_blocking).
int choose_bwd_threads(const fmb_view* views, int n_views, const long long* offs, int min_blocks, bool even_blocks) {
  const int cand[] = {128, 160};
  int best = 160;
  double best_cost = -1.0;
  for (int T : cand) {
    double cost = 0.0;
    for (int i = 0; i < n_views; ++i) {
      const int K = static_cast<int>(offs[views[i].object + 1] - offs[views[i].object]);
      const BwdBlocking b = bwd_blocking(K, T, min_blocks, even_blocks);
      cost += static_cast<double>(view_entries(views[i])) * (K / bwd_lane_fill(K, T, b.n_gb) + 5.0 * b.n_gb);
    }
    if (best_cost < 0.0 || cost < best_cost - 1e-9 || (std::fabs(cost - best_cost) <= 1e-9 && T > best)) {
      best_cost = cost;
      best = T;
    }
  }
  return best;
}

struct Plan {
  // A call's launches, one batch per launch: up to 64 views per batch, or (`big`: a
  // two-parameter call with more than 64 views) up to 256 in the *_big lists.
  bool big = false;
  std::vector<fmb::Batch> fwd;  // forward launches (tiles of rays)
  std::vector<fmb::Batch> bwd;  // backward launches (ray tiles x Gaussian blocks)
  std::vector<fmb::BigBatch> fwd_big, bwd_big, fmerge_big;
  long long n_records = 0;
  long long part_floats = 0;
  long long pair_stride = 0;  // stored-intermediate mode: floats per per-pair array
  long long n_gauss = 0;
  int maxK = 0;
  int rpt = kDefaultRpt;
  int ray_tile = 480;
  int bwd_threads = 160;
  int ac_run = 1;  // alpha compositing: forward rays per warp
  int ksplit = 1;  // two-parameter forward: Gaussian splits per view (1 = unsplit)
  long long fwd_part_floats = 0;  // split forward: per-ray partial sums
  std::vector<fmb::Batch> fmerge;  // split forward: merge launches (one per forward launch)
  long long n_entries = 0;         // plane entries of the batch (pixels or rays)
};

fmb_status validate_scene(const fmb_params* p, int n_objects, const long long* offs, int n_views,
                          const fmb_view* views) {
  if (!p) return fail(FMB_ERR_INVALID_ARG, "params is NULL");
  if (!std::isfinite(p->beta1) || !std::isfinite(p->beta2)) return fail(FMB_ERR_INVALID_ARG, "beta1/beta2 not finite");
  if (!(p->eta > 0.0f) || !std::isfinite(p->eta)) return fail(FMB_ERR_INVALID_ARG, "eta must be > 0");
  if (p->variant != 0 && p->variant != 1)
    return fail(FMB_ERR_INVALID_ARG, "variant must be 0 (two-parameter model) or 1 (alpha compositing)");
  if (p->variant == 1 && p->store_pairs)
    return fail(FMB_ERR_INVALID_ARG, "store_pairs is not available with variant 1 (alpha compositing)");
  if (p->n_flow < 0 || p->n_flow > 2) return fail(FMB_ERR_INVALID_ARG, "n_flow must be 0, 1 or 2");
  if (p->use_persistent != 0 && p->use_persistent != 1) return fail(FMB_ERR_INVALID_ARG, "use_persistent must be 0 or 1");
  if (p->store_pairs != 0 && p->store_pairs != 1) return fail(FMB_ERR_INVALID_ARG, "store_pairs must be 0 or 1");
  if (p->colors != 0 && p->colors != 1) return fail(FMB_ERR_INVALID_ARG, "colors must be 0 or 1");
  if (p->keep_order != 0 && p->keep_order != 1) return fail(FMB_ERR_INVALID_ARG, "keep_order must be 0 or 1");
  if (p->keep_order && p->variant != 1)
    return fail(FMB_ERR_INVALID_ARG, "keep_order applies to variant 1 (alpha compositing) only");
  if (p->colors && p->store_pairs) return fail(FMB_ERR_INVALID_ARG, "colors is not available with store_pairs");
  if (p->store_pairs && (p->fwd_rays_per_thread == 1 || p->fwd_rays_per_thread == 4))
    return fail(FMB_ERR_INVALID_ARG, "store_pairs needs fwd_rays_per_thread 0 or 2");
  if (p->fwd_rays_per_thread != 0 && p->fwd_rays_per_thread != 1 && p->fwd_rays_per_thread != 2 &&
      p->fwd_rays_per_thread != 4)
    return fail(FMB_ERR_INVALID_ARG, "fwd_rays_per_thread must be 0, 1, 2 or 4");
  if (p->fwd_threads != 0 && p->fwd_threads != 128) return fail(FMB_ERR_INVALID_ARG, "fwd_threads must be 0 or 128");
  if (p->fwd_ksplit < 0 || p->fwd_ksplit > 8) return fail(FMB_ERR_INVALID_ARG, "fwd_ksplit must be in [0, 8]");
  if (p->bwd_ray_tile != 0 && (p->bwd_ray_tile < 32 || p->bwd_ray_tile > 1024))
    return fail(FMB_ERR_INVALID_ARG, "bwd_ray_tile must be in [32, 1024] (0 = default)");
  if (p->bwd_threads != 0 && (p->bwd_threads < 32 || p->bwd_threads > 160 || (p->bwd_threads % 32) != 0))
    return fail(FMB_ERR_INVALID_ARG, "bwd_threads must be a multiple of 32 in [32, 160] (0 = default)");
  if (p->bwd_gblocks < 0 || p->bwd_gblocks > 64)
    return fail(FMB_ERR_INVALID_ARG, "bwd_gblocks must be in [0, 64] (0 = automatic)");
  if (n_objects < 1) return fail(FMB_ERR_INVALID_ARG, "n_objects must be >= 1");
  if (!offs) return fail(FMB_ERR_INVALID_ARG, "h_obj_offsets is NULL");
  if (offs[0] != 0) return fail(FMB_ERR_INVALID_ARG, "h_obj_offsets[0] must be 0");
  for (int k = 0; k < n_objects; ++k) {
    const long long K = offs[k + 1] - offs[k];
    if (K < 1) return fail(FMB_ERR_INVALID_ARG, "object " + std::to_string(k) + " has no Gaussians");
    if (K > kMaxK) return fail(FMB_ERR_INVALID_ARG, "object " + std::to_string(k) + " has too many Gaussians");
    if (p->variant == 1 && K > kMaxKAlphaCompositing)
      return fail(FMB_ERR_INVALID_ARG, "object " + std::to_string(k) +
                                           " has more than 256 Gaussians (the alpha-compositing limit)");
  }
  if (offs[n_objects] > kMaxGaussians) return fail(FMB_ERR_INVALID_ARG, "too many Gaussians in all");
  if (n_views < 1) return fail(FMB_ERR_INVALID_ARG, "n_views must be >= 1");
  if (!views) return fail(FMB_ERR_INVALID_ARG, "h_views is NULL");
  return FMB_OK;
}

fmb_status validate_views(int n_objects, int n_poses, int n_views, const fmb_view* views) {
  std::vector<std::pair<long long, long long>> spans;
  spans.reserve(n_views);
  for (int i = 0; i < n_views; ++i) {
    const fmb_view& v = views[i];
    const std::string id = "view " + std::to_string(i) + ": ";
    if (v.W < 1 || v.H < 1) return fail(FMB_ERR_INVALID_ARG, id + "W and H must be >= 1");
    if (static_cast<long long>(v.W) * v.H > (1ll << 30)) return fail(FMB_ERR_INVALID_ARG, id + "image too large");
    if (!(v.fx > 0.f) || !(v.fy > 0.f) || !std::isfinite(v.fx) || !std::isfinite(v.fy))
      return fail(FMB_ERR_INVALID_ARG, id + "fx, fy must be > 0");
    if (!std::isfinite(v.cx) || !std::isfinite(v.cy)) return fail(FMB_ERR_INVALID_ARG, id + "cx, cy not finite");
    if (v.object < 0 || v.object >= n_objects) return fail(FMB_ERR_INVALID_ARG, id + "object out of range");
    if (v.pose < 0 || v.pose >= n_poses) return fail(FMB_ERR_INVALID_ARG, id + "pose out of range");
    for (int j = 0; j < 2; ++j)
      if (v.flow_target[j] < -1 || v.flow_target[j] >= n_poses)
        return fail(FMB_ERR_INVALID_ARG, id + "flow_target out of range");
    if (v.pix_offset < 0) return fail(FMB_ERR_INVALID_ARG, id + "pix_offset < 0");
    if (v.rays != nullptr && v.n_rays < 1) return fail(FMB_ERR_INVALID_ARG, id + "n_rays must be >= 1 with rays");
    spans.emplace_back(v.pix_offset, v.pix_offset + view_entries(v));
  }
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i)
    if (spans[i].first < spans[i - 1].second) return fail(FMB_ERR_INVALID_ARG, "views overlap in the output planes");
  return FMB_OK;
}

template <class B, class Cost, class Count>
void order_items(B& b, Cost cost, Count count) {
  std::vector<int> idx(b.n_views);
  for (int i = 0; i < b.n_views; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(b.v[x]) > cost(b.v[y]); });
  long long acc = 0;
  for (int j = 0; j < b.n_views; ++j) {
    b.order_view[j] = idx[j];
    b.order_begin[j] = static_cast<int>(acc);
    acc += count(b.v[idx[j]]);
  }
  b.order_begin[b.n_views] = static_cast<int>(acc);
  b.n_items = static_cast<int>(acc);
}

// The views in batches of up to B::kCapacity, one batch per launch: each view's
// per-launch record (forward and backward tiling), the running offsets of its
// records, partial slots and stored pairs, and the batch's work items in cost order.
template <class B>
void fill_batches(Plan& pl, const fmb_params* p, const long long* offs, int n_views, const fmb_view* views, bool ac,
                  int rays_fwd, std::vector<B>& fwd, std::vector<B>& bwd, std::vector<B>& fmerge, long long& rec,
                  long long& part, long long& pairs) {
  const int n_flow = p->n_flow;
  for (int base = 0; base < n_views; base += B::kCapacity) {
    const int nb = std::min(B::kCapacity, n_views - base);
    B bf;
    std::memset(&bf, 0, sizeof(bf));
    B bb = bf;
    bf.n_views = bb.n_views = nb;
    long long ctas_f = 0, ctas_b = 0;
    for (int i = 0; i < nb; ++i) {
      const fmb_view& v = views[base + i];
      fmb::DevView d;
      std::memset(&d, 0, sizeof(d));
      d.W = v.W;
      d.H = v.H;
      d.fx = v.fx;
      d.fy = v.fy;
      d.cx = v.cx;
      d.cy = v.cy;
      d.pose = v.pose;
      d.tgt0 = n_flow > 0 ? v.flow_target[0] : -1;
      d.tgt1 = n_flow > 1 ? v.flow_target[1] : -1;
      d.K = static_cast<int>(offs[v.object + 1] - offs[v.object]);
      pl.maxK = std::max(pl.maxK, d.K);
      d.gauss_off = static_cast<int>(offs[v.object]);
      if (rec + d.K > kMaxRecords) throw std::runtime_error("too many (view, Gaussian) pairs in one batch");
      d.rec_off = static_cast<int>(rec);
      d.pix_off = v.pix_offset;
      rec += d.K;
      const long long P = view_entries(v);
      pl.n_entries += P;
      d.rays = v.rays;
      d.P = static_cast<int>(P);
      d.Kp = (d.K + 3) / 4 * 4;  // rows of 16-byte multiples
      d.pair_off = pairs;
      pairs += P * d.Kp;
      // forward
      fmb::DevView df = d;
      df.n_tiles = static_cast<int>((P + rays_fwd - 1) / rays_fwd);
      {
        // split s renders Gaussians [s GB, min(K, (s + 1) GB)); every split is non-empty
        const int S0 = std::min(pl.ksplit, d.K);
        df.GB = (d.K + S0 - 1) / S0;
        df.n_gblocks = (d.K + df.GB - 1) / df.GB;
        df.S = df.n_gblocks;
        df.part_off = pl.fwd_part_floats;
        if (df.n_gblocks > 1) pl.fwd_part_floats += 8 * P * df.n_gblocks;
      }
      ctas_f += static_cast<long long>(df.n_tiles) * df.n_gblocks;
      bf.v[i] = df;
      // backward
      fmb::DevView db = d;
      BwdBlocking bk = bwd_blocking(d.K, pl.bwd_threads, p->bwd_gblocks, p->store_pairs != 0);
      if (ac) bk = BwdBlocking{1, d.K, 1};  // one 32-ray tile x all K Gaussians per item
      const int tile_b = ac ? fmb::ac_rays_per_item() : pl.ray_tile;
      db.n_tiles = static_cast<int>((P + tile_b - 1) / tile_b);
      // two-parameter model: the view's rays spread evenly over its tiles (a
      // 500-ray view runs as two tiles of 250, not 320 + 180)
      db.rt = ac || db.n_tiles == 0 ? 0 : static_cast<int>((P + db.n_tiles - 1) / db.n_tiles);
      db.n_gblocks = bk.n_gb;
      db.GB = bk.GB;
      db.S = bk.S;
      db.slot_floats = (p->colors ? 13 : 10) * bk.GB + 12 * (1 + n_flow);
      db.part_off = part;
      part += static_cast<long long>(db.n_tiles) * db.n_gblocks * db.slot_floats;
      ctas_b += static_cast<long long>(db.n_tiles) * db.n_gblocks;
      bb.v[i] = db;
    }
    if (ctas_f > 0x7fffffffll || ctas_b > 0x7fffffffll) throw std::runtime_error("grid too large");
    // Work items view by view, the views ordered by decreasing cost per item
    // (forward: K x rays per tile; backward: Gaussians per block x rays per tile).
    order_items(bf, [&](const fmb::DevView& v) { return static_cast<double>(v.GB); },
                [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles) * v.n_gblocks; });
    if (pl.ksplit > 1) {
      // the merge: one item per tile of forward_merge_rays_per_item() rays of a view
      B bm = bf;
      const int rm = fmb::forward_merge_rays_per_item();
      for (int i = 0; i < nb; ++i) {
        // views left unsplit (fewer Gaussians than splits) were finished by the forward
        bm.v[i].n_tiles = bm.v[i].S > 1 ? (bm.v[i].P + rm - 1) / rm : 0;
        bm.v[i].n_gblocks = 1;
      }
      order_items(bm, [&](const fmb::DevView& v) { return static_cast<double>(v.S); },
                  [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles); });
      fmerge.push_back(bm);
    }
    order_items(bb, [&](const fmb::DevView& v) { return static_cast<double>(v.GB); },
                [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles) * v.n_gblocks; });
    fwd.push_back(bf);
    bwd.push_back(bb);
  }
}

// allow_big: the caller launches through the overloads that take 256-view batches
// (the two-parameter render and adjoint); others always get 64-view batches.
Plan make_plan(const fmb_params* p, const long long* offs, int n_objects, int n_views, const fmb_view* views,
               bool allow_big = false) {
  Plan pl;
  pl.rpt = p->fwd_rays_per_thread > 0 ? p->fwd_rays_per_thread : kDefaultRpt;
  pl.bwd_threads = p->bwd_threads > 0 ? p->bwd_threads : choose_bwd_threads(views, n_views, offs, p->bwd_gblocks, p->store_pairs != 0);
  // default ray tile: three rays per thread in the per-ray phase (balanced, and long
  // enough to amortise the per-CTA reductions)
  pl.ray_tile = p->bwd_ray_tile > 0 ? p->bwd_ray_tile : 3 * pl.bwd_threads;
  pl.n_gauss = offs[n_objects];
  const bool ac = p->variant == 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();  // no device (a host-only size query): plan for 152 SMs
    sms = 152;
  }
  if (ac) {
    long long total = 0;
    for (int i = 0; i < n_views; ++i) total += view_entries(views[i]);
    pl.ac_run = fmb::ac_fwd_run(total, sms);
  }
  const int rays_fwd = ac ? fmb::ac_fwd_rays_per_item(pl.ac_run) : fmb::forward_rays_per_cta(pl.rpt);
  // Gaussian split of the two-parameter forward: when the batch's ray tiles fill
  // less than half a wave of the GPU (about 6 resident forward CTAs per SM) and the
  // objects are large (K >= 128, so each CTA's serial Gaussian loop is long), each
  // tile's Gaussians are spread over enough CTAs for about 1.25 waves, at most 6.
  // Measured on the GB300: a 50 000-ray minibatch at K = 256 (200 tiles) 78.9 us
  // unsplit, 45.3 / 43.3 / 42.5 / 42.4 / 45.3 us with 4 / 5 / 6 / 7 / 8 splits,
  // while a single 320x240 view at K = 100 (300 tiles), a 64x64 view at K = 40 and
  // a 640x480 view at K = 256 (1200 tiles) only lose from splitting.
  if (!ac && !p->colors && !p->store_pairs && pl.rpt % 2 == 0 && p->fwd_ksplit != 1) {
    if (p->fwd_ksplit > 1) {
      pl.ksplit = p->fwd_ksplit;
    } else {
      long long tiles = 0;
      int maxK = 1;
      for (int i = 0; i < n_views; ++i) {
        tiles += (view_entries(views[i]) + rays_fwd - 1) / rays_fwd;
        maxK = std::max(maxK, static_cast<int>(offs[views[i].object + 1] - offs[views[i].object]));
      }
      const long long wave = static_cast<long long>(std::max(sms, 1)) * 6;
      if (tiles > 0 && 2 * tiles < wave && maxK >= 128) {
        const long long k = (wave + wave / 4 + tiles - 1) / tiles;
        pl.ksplit = static_cast<int>(std::max(1ll, std::min({k, 6ll, static_cast<long long>(maxK / 16)})));
      }
    }
  }
  long long rec = 0, part = 0, pairs = 0;
  // two-parameter calls with more than 64 views: one launch per pass for up to 256
  pl.big = allow_big && !ac && n_views > fmb::kMaxBatchViews;
  if (pl.big)
    fill_batches(pl, p, offs, n_views, views, ac, rays_fwd, pl.fwd_big, pl.bwd_big, pl.fmerge_big, rec, part, pairs);
  else
    fill_batches(pl, p, offs, n_views, views, ac, rays_fwd, pl.fwd, pl.bwd, pl.fmerge, rec, part, pairs);
  pl.n_records = rec;
  pl.part_floats = part;
  pl.pair_stride = (pairs + 63) / 64 * 64;
  if (p->store_pairs) pl.rpt = 2;
  return pl;
}

// Workspace: header (status word, work counters) | records | colour records (if
// colors) | deterministic partials (if deterministic) | per-pair t, e2, delta
// arrays (if store_pairs).
size_t crec_offset(const Plan& pl) {
  return kHeaderBytes + align256(static_cast<size_t>(pl.n_records) * 16 * fmb::kRecFloat4);
}
size_t partials_offset(const fmb_params* p, const Plan& pl) {
  return crec_offset(pl) + (p->colors ? align256(static_cast<size_t>(pl.n_records) * 16) : 0);
}
size_t pairs_offset(const fmb_params* p, const Plan& pl) {
  size_t bytes = partials_offset(p, pl);
  if (p->deterministic) bytes += align256(static_cast<size_t>(pl.part_floats) * sizeof(float));
  return bytes;
}

size_t fwd_part_offset(const fmb_params* p, const Plan& pl) {
  size_t bytes = pairs_offset(p, pl);
  if (p->store_pairs) bytes += align256(3 * static_cast<size_t>(pl.pair_stride) * sizeof(float));
  return bytes;
}

size_t order_offset(const fmb_params* p, const Plan& pl) {
  return fwd_part_offset(p, pl) + align256(static_cast<size_t>(pl.fwd_part_floats) * sizeof(float));
}

// keep_order: 32 M bytes (M of the alpha-compositing kernels) per plane entry.
size_t order_bytes(const fmb_params* p, const Plan& pl) {
  if (!p->keep_order) return 0;
  return align256(static_cast<size_t>(pl.n_entries) * 32 * fmb::ac_lanes_per_ray_elements(pl.maxK));
}

size_t workspace_needed(const fmb_params* p, const Plan& pl) { return order_offset(p, pl) + order_bytes(p, pl); }

fmb::Consts make_consts(const fmb_params* p) {
  const double log2e = 1.4426950408889634;
  fmb::Consts c;
  c.K2 = static_cast<float>(-(static_cast<double>(p->beta2) / p->eta) * log2e);
  c.K3 = static_cast<float>(-0.5 * log2e);
  c.beta1 = p->beta1;
  c.b2e = static_cast<float>(static_cast<double>(p->beta2) / p->eta);
  return c;
}

fmb_status check_workspace(void* ws, size_t bytes, size_t need) {
  if (!ws) return fail(FMB_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FMB_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < need)
    return fail(FMB_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                       std::to_string(bytes));
  return FMB_OK;
}

fmb_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FMB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

void fmb_default_params(fmb_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->beta1 = 21.4f;
  p->beta2 = 3.14f;
  p->eta = 1.0f;
  p->want_normals = 1;
  p->n_flow = 1;
}

const char* fmb_last_error(void) { return g_err.c_str(); }

const char* fmb_version(void) { return "fmb-gb300 0.1 (sm_103a)"; }

int fmb_forward_ksplit(const fmb_params* params, int n_objects, const long long* h_obj_offsets, int n_views,
                       const fmb_view* h_views) {
  try {
    if (validate_scene(params, n_objects, h_obj_offsets, n_views, h_views) != FMB_OK) return 0;
    return make_plan(params, h_obj_offsets, n_objects, n_views, h_views).ksplit;
  } catch (const std::exception& e) {
    fail(FMB_ERR_INVALID_ARG, e.what());
    return 0;
  }
}

int fmb_launch_count(const fmb_params* params, int n_objects, const long long* h_obj_offsets, int n_views,
                     const fmb_view* h_views, int pass, int want_pose) {
  try {
    if (validate_scene(params, n_objects, h_obj_offsets, n_views, h_views) != FMB_OK) return -1;
    if (pass != 0 && pass != 1) {
      fail(FMB_ERR_INVALID_ARG, "pass must be 0 (forward) or 1 (backward)");
      return -1;
    }
    const Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views, true);
    const int nb = static_cast<int>(pass == 0 ? (pl.big ? pl.fwd_big.size() : pl.fwd.size())
                                              : (pl.big ? pl.bwd_big.size() : pl.bwd.size()));
    if (pass == 0) return nb * (2 + (params->variant == 0 && pl.ksplit > 1 ? 1 : 0));  // prologue, forward, merge
    if (nb == 0) return 1;  // the zeroing launch
    // prologue and backward per batch; deterministic mode adds the Gaussian (and pose) reductions
    return nb * (2 + (params->deterministic ? 1 + (want_pose ? 1 : 0) : 0));
  } catch (const std::exception& e) {
    fail(FMB_ERR_INVALID_ARG, e.what());
    return -1;
  }
}

size_t fmb_workspace_bytes(const fmb_params* params, int n_objects, const long long* h_obj_offsets, int n_views,
                           const fmb_view* h_views) {
  try {
    if (validate_scene(params, n_objects, h_obj_offsets, n_views, h_views) != FMB_OK) return 0;
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views);
    return workspace_needed(params, pl);
  } catch (const std::exception& e) {
    fail(FMB_ERR_INVALID_ARG, e.what());
    return 0;
  } catch (...) {
    fail(FMB_ERR_INVALID_ARG, "unknown error");
    return 0;
  }
}

fmb_status fmb_render_forward(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                              const float* means, const float* chol, const float* weights, const float* colors,
                              int n_poses, const float* poses, int n_views, const fmb_view* h_views,
                              float* depth, float* alpha, float* normal, float* flow, float* color, float* saved,
                              void* workspace, size_t workspace_bytes, fmb_stream_t stream) {
  try {
    g_err.clear();
    fmb_status st = validate_scene(params, n_objects, h_obj_offsets, n_views, h_views);
    if (st != FMB_OK) return st;
    if (n_poses < 1 || !poses) return fail(FMB_ERR_INVALID_ARG, "poses missing");
    if (!means || !chol || !weights) return fail(FMB_ERR_INVALID_ARG, "means, chol and weights are required");
    if (!depth || !alpha || !saved) return fail(FMB_ERR_INVALID_ARG, "depth, alpha and saved are required");
    if (params->want_normals && !normal) return fail(FMB_ERR_INVALID_ARG, "normal is NULL but want_normals is set");
    if (params->n_flow > 0 && !flow) return fail(FMB_ERR_INVALID_ARG, "flow is NULL but n_flow > 0");
    if (params->colors && (!colors || !color))
      return fail(FMB_ERR_INVALID_ARG, "colors and color are required when params->colors is set");
    st = validate_views(n_objects, n_poses, n_views, h_views);
    if (st != FMB_OK) return st;
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views, true);
    st = check_workspace(workspace, workspace_bytes, workspace_needed(params, pl));
    if (st != FMB_OK) return st;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(workspace);
    float4* records = reinterpret_cast<float4*>(static_cast<char*>(workspace) + kHeaderBytes);
    fmb::Scene sc{means, chol, weights, poses};
    if (params->colors) {
      sc.colors = colors;
      sc.crec = reinterpret_cast<float4*>(static_cast<char*>(workspace) + crec_offset(pl));
    }
    if (!params->colors) color = nullptr;
    const fmb::Consts c = make_consts(params);
    float* pairs = params->store_pairs
                       ? reinterpret_cast<float*>(static_cast<char*>(workspace) + pairs_offset(params, pl))
                       : nullptr;
    cudaError_t e = cudaSuccess;
    int* counter = params->use_persistent
                       ? reinterpret_cast<int*>(reinterpret_cast<char*>(status) + kFwdCounterOffset)
                       : nullptr;
    // batches: pl.fwd / pl.fmerge, or their 256-view counterparts
    auto run = [&](const auto& fwd, const auto& fmerge) -> fmb_status {
      for (size_t bi = 0; bi < fwd.size(); ++bi) {
        const auto& b = fwd[bi];
        e = fmb::launch_prologue(b, sc, c, records, pl.maxK, bi == 0 ? status : nullptr, counter, s);
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        fmb::FwdOut fo{depth, alpha, normal, flow, saved, pairs, pl.pair_stride};
        fo.color = color;
        fo.part = reinterpret_cast<float*>(static_cast<char*>(workspace) + fwd_part_offset(params, pl));
        if (params->keep_order) fo.order = static_cast<unsigned char*>(workspace) + order_offset(params, pl);
        if constexpr (std::is_same_v<std::decay_t<decltype(b)>, fmb::Batch>) {
          if (params->variant == 1) {  // alpha compositing: 64-view batches only
            fo.pairs = nullptr;
            e = fmb::launch_forward_ac(b, sc, c, records, params->want_normals != 0, params->n_flow, pl.maxK, fo,
                                       pl.ac_run, status, counter, s);
            if (e != cudaSuccess) return cuda_fail(e, "forward launch");
            continue;
          }
        }
        e = fmb::launch_forward(b, sc, c, records, params->want_normals != 0, params->n_flow, pl.rpt, pl.maxK, fo,
                                status, counter, s);
        if (e == cudaSuccess && pl.ksplit > 1)
          e = fmb::launch_forward_merge(fmerge[bi], sc, params->want_normals != 0, params->n_flow, fo, s);
        if (e != cudaSuccess) return cuda_fail(e, "forward launch");
      }
      return FMB_OK;
    };
    return pl.big ? run(pl.fwd_big, pl.fmerge_big) : run(pl.fwd, pl.fmerge);
  } catch (const std::exception& e) {
    return fail(FMB_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return fail(FMB_ERR_INVALID_ARG, "unknown error");
  }
}

fmb_status fmb_render_backward(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                               const float* means, const float* chol, const float* weights, const float* colors,
                               int n_poses, const float* poses, int n_views, const fmb_view* h_views,
                               const float* depth, const float* normal, const float* color, const float* saved,
                               const float* g_depth, const float* g_alpha, const float* g_normal,
                               const float* g_flow, const float* g_color, float* grad_means, float* grad_chol,
                               float* grad_weights, float* grad_colors, float* grad_poses, void* workspace,
                               size_t workspace_bytes, fmb_stream_t stream) {
  try {
    g_err.clear();
    fmb_status st = validate_scene(params, n_objects, h_obj_offsets, n_views, h_views);
    if (st != FMB_OK) return st;
    if (n_poses < 1 || !poses) return fail(FMB_ERR_INVALID_ARG, "poses missing");
    if (!means || !chol || !weights) return fail(FMB_ERR_INVALID_ARG, "means, chol and weights are required");
    if (!depth || !saved) return fail(FMB_ERR_INVALID_ARG, "depth and saved (forward outputs) are required");
    if (params->want_normals && g_normal && !normal)
      return fail(FMB_ERR_INVALID_ARG, "normal (forward output) is required with g_normal");
    if (!grad_means || !grad_chol || !grad_weights)
      return fail(FMB_ERR_INVALID_ARG, "grad_means, grad_chol and grad_weights are required");
    if (params->colors && (!colors || !color || !grad_colors))
      return fail(FMB_ERR_INVALID_ARG, "colors, color and grad_colors are required when params->colors is set");
    st = validate_views(n_objects, n_poses, n_views, h_views);
    if (st != FMB_OK) return st;
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views, true);
    st = check_workspace(workspace, workspace_bytes, workspace_needed(params, pl));
    if (st != FMB_OK) return st;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(workspace);
    char* base = static_cast<char*>(workspace);
    float4* records = reinterpret_cast<float4*>(base + kHeaderBytes);
    float* partials = nullptr;
    if (params->deterministic) partials = reinterpret_cast<float*>(base + partials_offset(params, pl));
    fmb::Scene sc{means, chol, weights, poses};
    if (params->colors) {
      sc.colors = colors;
      sc.crec = reinterpret_cast<float4*>(base + crec_offset(pl));
    }
    const fmb::Consts c = make_consts(params);
    const bool normals = params->want_normals != 0;
    const float* pairs =
        params->store_pairs ? reinterpret_cast<const float*>(base + pairs_offset(params, pl)) : nullptr;
    fmb::BwdIn in{depth,   normals ? normal : nullptr, saved, g_depth, g_alpha, normals ? g_normal : nullptr,
                  params->n_flow > 0 ? g_flow : nullptr, pairs, pl.pair_stride};
    fmb::BwdOut out{grad_means, grad_chol, grad_weights, grad_poses, partials};
    if (params->colors) {
      in.color = color;
      in.g_color = g_color;
      out.gcolors = grad_colors;
    }
    if (params->keep_order) in.order = reinterpret_cast<const unsigned char*>(base + order_offset(params, pl));

    fmb::ZeroJob zj{};
    zj.ptr[0] = reinterpret_cast<float*>(status);
    zj.n[0] = 1;
    zj.ptr[1] = grad_means;
    zj.n[1] = 3 * pl.n_gauss;
    zj.ptr[2] = grad_chol;
    zj.n[2] = 6 * pl.n_gauss;
    zj.ptr[3] = grad_weights;
    zj.n[3] = pl.n_gauss;
    zj.ptr[4] = grad_poses;
    zj.n[4] = grad_poses ? 12ll * n_poses : 0;
    zj.ptr[5] = params->colors ? grad_colors : nullptr;
    zj.n[5] = params->colors ? 3 * pl.n_gauss : 0;
    cudaError_t e = cudaSuccess;
    int* counter = params->use_persistent ? reinterpret_cast<int*>(base + kBwdCounterOffset) : nullptr;
    bool first = true;  // the first batch's prologue clears the outputs and the status word
    // batches: pl.bwd, or its 256-view counterpart
    auto run = [&](const auto& bwd) -> fmb_status {
      for (const auto& b : bwd) {
        e = fmb::launch_prologue(b, sc, c, records, pl.maxK, nullptr, counter, s, first ? &zj : nullptr);
        first = false;
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        bool done = false;
        if constexpr (std::is_same_v<std::decay_t<decltype(b)>, fmb::Batch>) {
          if (params->variant == 1) {  // alpha compositing: 64-view batches only
            e = fmb::launch_backward_ac(b, sc, c, records, normals, params->n_flow, pl.maxK, in, out, status,
                                        counter, s);
            done = true;
          }
        }
        if (!done)
          e = fmb::launch_backward(b, sc, c, records, normals, params->n_flow, pl.ray_tile, pl.bwd_threads, in, out,
                                   counter, s);
        if (e != cudaSuccess) return cuda_fail(e, "backward launch");
        if (partials) {
          e = fmb::launch_backward_reduce(b, params->n_flow, pl.n_gauss, n_poses, out, s);
          if (e != cudaSuccess) return cuda_fail(e, "reduction launch");
        }
      }
      return FMB_OK;
    };
    st = pl.big ? run(pl.bwd_big) : run(pl.bwd);
    if (st != FMB_OK) return st;
    if (first) {  // nothing to render: the outputs are still cleared
      e = fmb::launch_zero(zj, s);
      if (e != cudaSuccess) return cuda_fail(e, "zeroing launch");
    }
    return FMB_OK;
  } catch (const std::exception& e) {
    return fail(FMB_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return fail(FMB_ERR_INVALID_ARG, "unknown error");
  }
}

fmb_status fmb_render_points(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                             const float* means, const float* chol, const float* weights, int n_poses,
                             const float* poses, int n_views, const fmb_view* h_views, const float* depth,
                             const float* saved, float* points, float* normal_tf, float* normal_screen,
                             float* quality, void* workspace, size_t workspace_bytes, fmb_stream_t stream) {
  try {
    g_err.clear();
    fmb_status st = validate_scene(params, n_objects, h_obj_offsets, n_views, h_views);
    if (st != FMB_OK) return st;
    if (n_poses < 1 || !poses) return fail(FMB_ERR_INVALID_ARG, "poses missing");
    if (!means || !chol || !weights) return fail(FMB_ERR_INVALID_ARG, "means, chol and weights are required");
    if (!depth || !saved) return fail(FMB_ERR_INVALID_ARG, "depth and saved (forward outputs) are required");
    st = validate_views(n_objects, n_poses, n_views, h_views);
    if (st != FMB_OK) return st;
    if (normal_screen != nullptr)
      for (int i = 0; i < n_views; ++i)
        if (h_views[i].rays != nullptr)
          return fail(FMB_ERR_INVALID_ARG, "normal_screen needs whole images (Eq. 16 takes image neighbours); "
                                           "pass NULL for ray batches");
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views);
    st = check_workspace(workspace, workspace_bytes, workspace_needed(params, pl));
    if (st != FMB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4* records = reinterpret_cast<float4*>(static_cast<char*>(workspace) + kHeaderBytes);
    const fmb::Scene sc{means, chol, weights, poses};
    const fmb::Consts c = make_consts(params);
    // alpha compositing: the forward's run of neighbouring rays per warp
    const int per = params->variant == 1 ? fmb::ac_fwd_rays_per_item(pl.ac_run) : fmb::points_rays_per_item();
    for (fmb::Batch b : pl.fwd) {
      for (int i = 0; i < b.n_views; ++i) b.v[i].n_tiles = (b.v[i].P + per - 1) / per;
      order_items(b, [&](const fmb::DevView& v) { return static_cast<double>(v.K); },
                  [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles); });
      cudaError_t e = fmb::launch_prologue(b, sc, c, records, pl.maxK, nullptr, nullptr, s);
      if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
      e = fmb::launch_points(b, sc, c, records, params->variant, pl.maxK, pl.ac_run, depth, saved, points, normal_tf,
                             normal_screen, quality, s);
      if (e != cudaSuccess) return cuda_fail(e, "points launch");
    }
    return FMB_OK;
  } catch (const std::exception& e) {
    return fail(FMB_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return fail(FMB_ERR_INVALID_ARG, "unknown error");
  }
}

fmb_status fmb_loss_attribution(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                                const float* means, const float* chol, const float* weights, int n_poses,
                                const float* poses, int n_views, const fmb_view* h_views, const float* saved,
                                const float* ray_loss, float* attribution, void* workspace, size_t workspace_bytes,
                                fmb_stream_t stream) {
  try {
    g_err.clear();
    fmb_status st = validate_scene(params, n_objects, h_obj_offsets, n_views, h_views);
    if (st != FMB_OK) return st;
    if (n_poses < 1 || !poses) return fail(FMB_ERR_INVALID_ARG, "poses missing");
    if (!means || !chol || !weights) return fail(FMB_ERR_INVALID_ARG, "means, chol and weights are required");
    if (!saved && params->variant != 1) return fail(FMB_ERR_INVALID_ARG, "saved (forward output) is required");
    if (!ray_loss || !attribution) return fail(FMB_ERR_INVALID_ARG, "ray_loss and attribution are required");
    st = validate_views(n_objects, n_poses, n_views, h_views);
    if (st != FMB_OK) return st;
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views);
    st = check_workspace(workspace, workspace_bytes, workspace_needed(params, pl));
    if (st != FMB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4* records = reinterpret_cast<float4*>(static_cast<char*>(workspace) + kHeaderBytes);
    const fmb::Scene sc{means, chol, weights, poses};
    const fmb::Consts c = make_consts(params);
    fmb::ZeroJob zj{};
    zj.ptr[0] = attribution;
    zj.n[0] = pl.n_gauss;
    cudaError_t e = cudaSuccess;
    bool first = true;  // the first batch's prologue clears the attribution output
    if (params->variant == 0) {
      // two-parameter model: the backward's blocking (two Gaussians per thread)
      const int T = pl.bwd_threads;
      const int tile = fmb::attribution2_ray_tile(T);
      for (fmb::Batch b : pl.fwd) {
        for (int i = 0; i < b.n_views; ++i) {
          const BwdBlocking bk = bwd_blocking(b.v[i].K, T);
          b.v[i].n_tiles = (b.v[i].P + tile - 1) / tile;
          b.v[i].n_gblocks = bk.n_gb;
          b.v[i].GB = bk.GB;
          b.v[i].S = bk.S;
        }
        order_items(b, [&](const fmb::DevView& v) { return static_cast<double>(v.GB); },
                    [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles) * v.n_gblocks; });
        e = fmb::launch_prologue(b, sc, c, records, pl.maxK, nullptr, nullptr, s, first ? &zj : nullptr);
        first = false;
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        e = fmb::launch_attribution2(b, sc, c, records, T, tile, saved, ray_loss, attribution, s);
        if (e != cudaSuccess) return cuda_fail(e, "attribution launch");
      }
    } else {
      const int per = fmb::attribution_rays_per_item();
      const int blk = 32 * (pl.maxK <= 64 ? 2 : (pl.maxK <= 128 ? 4 : 8));
      for (fmb::Batch b : pl.fwd) {
        for (int i = 0; i < b.n_views; ++i) {
          b.v[i].n_tiles = (b.v[i].P + per - 1) / per;
          b.v[i].n_gblocks = (b.v[i].K + blk - 1) / blk;
        }
        order_items(b, [&](const fmb::DevView& v) { return static_cast<double>(std::min(v.K, blk)); },
                    [](const fmb::DevView& v) { return static_cast<long long>(v.n_tiles) * v.n_gblocks; });
        e = fmb::launch_prologue(b, sc, c, records, pl.maxK, nullptr, nullptr, s, first ? &zj : nullptr);
        first = false;
        if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
        e = fmb::launch_attribution_ac(b, sc, c, records, pl.maxK, ray_loss, attribution, s);
        if (e != cudaSuccess) return cuda_fail(e, "attribution launch");
      }
    }
    if (first) {  // nothing to render: the output is still cleared
      e = fmb::launch_zero(zj, s);
      if (e != cudaSuccess) return cuda_fail(e, "zeroing launch");
    }
    return FMB_OK;
  } catch (const std::exception& e) {
    return fail(FMB_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return fail(FMB_ERR_INVALID_ARG, "unknown error");
  }
}

fmb_status fmb_read_device_status(const void* workspace, int* h_status, fmb_stream_t stream) {
  if (!workspace || !h_status) return fail(FMB_ERR_INVALID_ARG, "workspace and h_status are required");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h_status, workspace, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
  return FMB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------
// Forward render without a caller-provided workspace.
//
// Some callers cannot allocate device memory: a plugin whose host application
// owns all device memory and exposes no allocator, or code on a real-time path
// where cudaMalloc's implicit device synchronisation is not acceptable.  For them
// the forward pass's scratch (status word and per-(view, Gaussian) records) lives
// in the fixed array below, which every device that loads this library holds
// until the process exits.  No cudaMalloc, cudaFree or allocating library routine
// is called.
//
// The array's name is only a host-side stand-in: the device address is obtained
// once per device with cudaGetSymbolAddress, during that device's first call
// (so the first call on a device should come before any stream capture).  The
// address is cached for the life of the process: a device reset (or any other
// teardown of the device's primary context) invalidates it, and the entry point
// must not be used after one.  All calls share the array and it keeps the last
// call's contents; the status word is cleared by every call and the records are
// rewritten, but calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.  fmb_read_noalloc_status reads the status
// word back.

namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;  // 1 MiB
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_fmb_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {nullptr};

fmb_status static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(FMB_ERR_CUDA, "device index out of range for static scratch");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fmb_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return FMB_OK;
}

}  // namespace

extern "C" fmb_status fmb_render_forward_noalloc(const fmb_params* params, int n_objects,
                                                 const long long* h_obj_offsets, const float* means,
                                                 const float* chol, const float* weights, const float* colors,
                                                 int n_poses, const float* poses, int n_views,
                                                 const fmb_view* h_views, float* depth, float* alpha, float* normal,
                                                 float* flow, float* color, float* saved, fmb_stream_t stream) {
  try {
    g_err.clear();
    fmb_status st = validate_scene(params, n_objects, h_obj_offsets, n_views, h_views);
    if (st != FMB_OK) return st;
    if (n_poses < 1 || !poses) return fail(FMB_ERR_INVALID_ARG, "poses missing");
    if (!means || !chol || !weights) return fail(FMB_ERR_INVALID_ARG, "means, chol and weights are required");
    if (!depth || !alpha || !saved) return fail(FMB_ERR_INVALID_ARG, "depth, alpha and saved are required");
    if (params->want_normals && !normal) return fail(FMB_ERR_INVALID_ARG, "normal is NULL but want_normals is set");
    if (params->n_flow > 0 && !flow) return fail(FMB_ERR_INVALID_ARG, "flow is NULL but n_flow > 0");
    st = validate_views(n_objects, n_poses, n_views, h_views);
    if (st != FMB_OK) return st;
    if (params->store_pairs)
      return fail(FMB_ERR_INVALID_ARG, "store_pairs needs a workspace (use fmb_render_forward)");
    if (params->keep_order)
      return fail(FMB_ERR_INVALID_ARG, "keep_order needs a workspace (use fmb_render_forward)");
    fmb_params unsplit = *params;  // the fixed scratch holds the records only: no Gaussian split
    unsplit.fwd_ksplit = 1;
    params = &unsplit;
    Plan pl = make_plan(params, h_obj_offsets, n_objects, n_views, h_views);
    if (params->colors && (!colors || !color))
      return fail(FMB_ERR_INVALID_ARG, "colors and color are required when params->colors is set");
    const size_t need = partials_offset(params, pl);
    if (need > kStaticScratchBytes)
      return fail(FMB_ERR_WORKSPACE, "batch needs " + std::to_string(need) + " bytes of scratch; the static scratch " +
                                         "holds " + std::to_string(kStaticScratchBytes) +
                                         " (64 bytes per view and Gaussian, 80 with colours, plus 256)");
    void* ws = nullptr;
    st = static_scratch_address(&ws);
    if (st != FMB_OK) return st;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(ws);
    float4* records = reinterpret_cast<float4*>(static_cast<char*>(ws) + kHeaderBytes);
    fmb::Scene sc{means, chol, weights, poses};
    if (params->colors) {
      sc.colors = colors;
      sc.crec = reinterpret_cast<float4*>(static_cast<char*>(ws) + crec_offset(pl));
    }
    if (!params->colors) color = nullptr;
    const fmb::Consts c = make_consts(params);
    float* pairs = nullptr;  // stored-intermediate mode is rejected above
    cudaError_t e = cudaSuccess;
    int* counter = params->use_persistent
                       ? reinterpret_cast<int*>(reinterpret_cast<char*>(status) + kFwdCounterOffset)
                       : nullptr;
    for (size_t bi = 0; bi < pl.fwd.size(); ++bi) {
      const fmb::Batch& b = pl.fwd[bi];
      e = fmb::launch_prologue(b, sc, c, records, pl.maxK, bi == 0 ? status : nullptr, counter, s);
      if (e != cudaSuccess) return cuda_fail(e, "prologue launch");
      fmb::FwdOut fo{depth, alpha, normal, flow, saved, pairs, pl.pair_stride};
      fo.color = color;
      if (params->variant == 1) {
        fo.pairs = nullptr;
        e = fmb::launch_forward_ac(b, sc, c, records, params->want_normals != 0, params->n_flow, pl.maxK, fo, pl.ac_run,
                                   status, counter, s);
      } else {
        e = fmb::launch_forward(b, sc, c, records, params->want_normals != 0, params->n_flow, pl.rpt, pl.maxK, fo,
                                status, counter, s);
      }
      if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    }
    return FMB_OK;
  } catch (const std::exception& e) {
    return fail(FMB_ERR_INVALID_ARG, e.what());
  } catch (...) {
    return fail(FMB_ERR_INVALID_ARG, "unknown error");
  }
}

// Status word of the fixed scratch (its first int), copied to the host after the
// work already enqueued on `stream` (the caller's last allocation-free forward) has
// run.  Uses the same cached device address as the render call; no allocation.
extern "C" fmb_status fmb_read_noalloc_status(int* h_status, fmb_stream_t stream) {
  if (!h_status) return fail(FMB_ERR_INVALID_ARG, "h_status is required");
  void* ws = nullptr;
  fmb_status st = static_scratch_address(&ws);
  if (st != FMB_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h_status, ws, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the fixed scratch's status word");
  return FMB_OK;
}
