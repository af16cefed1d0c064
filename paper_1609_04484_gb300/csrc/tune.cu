// Autotuner of the pair kernels' launch shapes (not in the paper: the
// direct sum replaces the paper's FMM, and its best CTA shape depends on the
// problem size and the arithmetic).
//
// Each pair kernel is compiled in a few shape variants (threads per CTA,
// targets per thread, sources per shared-memory tile); the source range is
// further split so that the grid holds about 2, 4 or 8 CTAs per SM. The tuner
// times every (variant, split) combination on a handle with CUDA events on
// the handle's stream and keeps the fastest, both on the handle and in a
// process-wide cache keyed by (precision, ceil(log2 N), ceil(log2 T)), where N
// is the number of sources and T of targets. Later handles of the same size
// class pick the cached shape up without tuning. The cache can be written to
// and read from a file of JSON lines, one entry per line.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kCtasPerSm[] = {2, 4, 8};
constexpr int kMaxVariants = 16;

struct CacheEntry {
  int variant;
  int ctas_per_sm;
  double ms;
};
using CacheKey = std::tuple<int, int, int>;  // precision, ceil log2 N, ceil log2 T

std::mutex g_cache_mu;
std::map<CacheKey, CacheEntry> g_cache;

int ceil_log2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

int variants_of(int precision, PairVariant* out) {
  switch (precision) {
    case STOKES_FP64: return pair_variants_f64(out, kMaxVariants);
    case STOKES_FP32: return pair_variants_f32(out, kMaxVariants);
    case STOKES_DF64: return pair_variants_df64(out, kMaxVariants);
    default: throw Error(STOKES_EINVAL, "precision must be FP64, FP32 or DF64");
  }
}

bool valid_shape(int precision, int variant, int ctas_per_sm) {
  PairVariant v[kMaxVariants];
  const int n = variants_of(precision, v);
  return variant >= 0 && variant < n && ctas_per_sm >= 1 && ctas_per_sm <= 64;
}

// value of "key": <number> in a flat JSON object; false if absent
bool json_number(const std::string& line, const char* key, double& out) {
  const std::string pat = std::string("\"") + key + "\"";
  size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  p = line.find(':', p + pat.size());
  if (p == std::string::npos) return false;
  const char* s = line.c_str() + p + 1;
  char* end = nullptr;
  const double v = std::strtod(s, &end);
  if (end == s) return false;
  out = v;
  return true;
}

}  // namespace

PairShape pair_shape(const Geom& g, int precision, int64_t T) {
  if (precision >= 0 && precision < 3 && g.shape[precision].variant >= 0) return g.shape[precision];
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(CacheKey(precision, ceil_log2(g.N), ceil_log2(T)));
    if (it != g_cache.end()) return PairShape{it->second.variant, it->second.ctas_per_sm};
  }
  return PairShape{0, 4};
}

// Times every shape of the pair kernel of `precision` on the handle's nodes
// as targets (a zero density: the work per pair does not depend on it) and
// sets the fastest on the handle and in the cache. Returns it.
static PairShape autotune(Geom& g, int precision, int reps, double& best_ms) {
  require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64,
          "precision must be FP64, FP32 or DF64");
  require(reps >= 1 && reps <= 100, "reps must be in [1, 100]");
  PairVariant vars[kMaxVariants];
  const int nv = variants_of(precision, vars);
  cudaStream_t s = g.stream;
  DevBuf<double2> sig;
  sig.alloc(g.N);
  STOKES_CUDA(cudaMemsetAsync(sig.get(), 0, g.N * sizeof(double2), s));
  const bool prof_on = g.prof.on;
  g.prof.on = false;
  cudaEvent_t a = nullptr, b = nullptr;
  STOKES_CUDA(cudaEventCreate(&a));
  STOKES_CUDA(cudaEventCreate(&b));
  PairShape best{0, 4};
  best_ms = INFINITY;
  try {
    for (int v = 0; v < nv; ++v) {
      for (int cps : kCtasPerSm) {
        const PairShape sh{v, cps};
        auto launch = [&] {
          if (precision == STOKES_FP64) pairs_f64(g, sig.get(), g.pos.get(), g.N, true, sh, nullptr);
          else if (precision == STOKES_FP32) pairs_f32(g, sig.get(), g.pos.get(), g.N, sh, nullptr);
          else pairs_df64(g, sig.get(), g.pos.get(), g.N, sh, nullptr);
        };
        launch();  // warm-up (and the partial-sum buffer's growth)
        STOKES_CUDA(cudaEventRecord(a, s));
        for (int r = 0; r < reps; ++r) launch();
        STOKES_CUDA(cudaEventRecord(b, s));
        STOKES_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        STOKES_CUDA(cudaEventElapsedTime(&ms, a, b));
        const double per = (double)ms / reps;
        if (per < best_ms) {
          best_ms = per;
          best = sh;
        }
      }
    }
  } catch (...) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    g.prof.on = prof_on;
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g.prof.on = prof_on;
  g.shape[precision] = best;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache[CacheKey(precision, ceil_log2(g.N), ceil_log2(g.N))] = CacheEntry{best.variant, best.ctas_per_sm, best_ms};
  return best;
}

}  // namespace stokes


namespace {

template <class F>
int run(F&& f) {
  struct Ctx {
    F* f;
  } ctx{&f};
  return stokes::guarded_call([](void* c) { (*static_cast<Ctx*>(c)->f)(); }, &ctx);
}

}  // namespace

extern "C" {

int stokes_pair_shape_count(int precision) {
  stokes::PairVariant v[stokes::kMaxVariants];
  if (precision == STOKES_FP64) return stokes::pair_variants_f64(v, stokes::kMaxVariants);
  if (precision == STOKES_FP32) return stokes::pair_variants_f32(v, stokes::kMaxVariants);
  if (precision == STOKES_DF64) return stokes::pair_variants_df64(v, stokes::kMaxVariants);
  return STOKES_EINVAL;
}

int stokes_pair_shape_info(int precision, int variant, int* threads, int* targets_per_thread, int* tile) {
  return run([&] {
    stokes::PairVariant v[stokes::kMaxVariants];
    const int n = stokes::variants_of(precision, v);
    stokes::require(variant >= 0 && variant < n, "unknown shape variant");
    if (threads) *threads = v[variant].threads;
    if (targets_per_thread) *targets_per_thread = v[variant].tpt;
    if (tile) *tile = v[variant].tile;
  });
}

int stokes_set_pair_shape(stokes_geom* h, int precision, int variant, int ctas_per_sm) {
  return run([&] {
    stokes::require(h && h->g, "null handle");
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64,
                    "precision must be FP64, FP32 or DF64");
    if (variant < 0) {
      h->g->shape[precision] = stokes::PairShape{};
      return;
    }
    stokes::require(stokes::valid_shape(precision, variant, ctas_per_sm), "bad shape variant or ctas_per_sm");
    h->g->shape[precision] = stokes::PairShape{variant, ctas_per_sm};
  });
}

int stokes_get_pair_shape(stokes_geom* h, int precision, int64_t n_targets, int* variant, int* ctas_per_sm) {
  return run([&] {
    stokes::require(h && h->g, "null handle");
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64,
                    "precision must be FP64, FP32 or DF64");
    stokes::require(n_targets >= 1, "n_targets must be >= 1");
    const stokes::PairShape sh = stokes::pair_shape(*h->g, precision, n_targets);
    if (variant) *variant = sh.variant;
    if (ctas_per_sm) *ctas_per_sm = sh.ctas_per_sm;
  });
}

int stokes_autotune(stokes_geom* h, int precision, int reps, int* variant, int* ctas_per_sm, double* best_ms) {
  return run([&] {
    stokes::require(h && h->g, "null handle");
    double ms = 0.0;
    const stokes::PairShape sh = stokes::autotune(*h->g, precision, reps, ms);
    if (variant) *variant = sh.variant;
    if (ctas_per_sm) *ctas_per_sm = sh.ctas_per_sm;
    if (best_ms) *best_ms = ms;
  });
}

int stokes_tune_cache_insert(int precision, int64_t n_sources, int64_t n_targets, int variant, int ctas_per_sm,
                             double ms) {
  return run([&] {
    stokes::require(n_sources >= 1 && n_targets >= 1, "sizes must be >= 1");
    stokes::require(stokes::valid_shape(precision, variant, ctas_per_sm), "bad shape variant or ctas_per_sm");
    std::lock_guard<std::mutex> lk(stokes::g_cache_mu);
    stokes::g_cache[stokes::CacheKey(precision, stokes::ceil_log2(n_sources), stokes::ceil_log2(n_targets))] =
        stokes::CacheEntry{variant, ctas_per_sm, ms};
  });
}

int stokes_tune_cache_lookup(int precision, int64_t n_sources, int64_t n_targets, int* variant, int* ctas_per_sm,
                             double* ms) {
  return run([&] {
    stokes::require(n_sources >= 1 && n_targets >= 1, "sizes must be >= 1");
    std::lock_guard<std::mutex> lk(stokes::g_cache_mu);
    auto it = stokes::g_cache.find(
        stokes::CacheKey(precision, stokes::ceil_log2(n_sources), stokes::ceil_log2(n_targets)));
    const bool hit = it != stokes::g_cache.end();
    if (variant) *variant = hit ? it->second.variant : -1;
    if (ctas_per_sm) *ctas_per_sm = hit ? it->second.ctas_per_sm : 0;
    if (ms) *ms = hit ? it->second.ms : 0.0;
  });
}

int stokes_tune_cache_clear(void) {
  return run([&] {
    std::lock_guard<std::mutex> lk(stokes::g_cache_mu);
    stokes::g_cache.clear();
  });
}

int stokes_tune_cache_save(const char* path) {
  return run([&] {
    stokes::require(path && *path, "null path");
    std::lock_guard<std::mutex> lk(stokes::g_cache_mu);
    const std::string tmp = std::string(path) + ".tmp";
    {
      std::ofstream out(tmp);
      stokes::require((bool)out, std::string("cannot write ") + tmp);
      for (const auto& kv : stokes::g_cache) {
        stokes::PairVariant v[stokes::kMaxVariants];
        stokes::variants_of(std::get<0>(kv.first), v);
        const stokes::PairVariant& pv = v[kv.second.variant];
        char line[320];
        std::snprintf(line, sizeof line,
                      "{\"precision\": %d, \"log2_sources\": %d, \"log2_targets\": %d, \"variant\": %d, "
                      "\"threads\": %d, \"targets_per_thread\": %d, \"tile\": %d, \"ctas_per_sm\": %d, "
                      "\"ms\": %.6g}\n",
                      std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), kv.second.variant,
                      pv.threads, pv.tpt, pv.tile, kv.second.ctas_per_sm, kv.second.ms);
        out << line;
      }
      stokes::require((bool)out, std::string("write failed: ") + tmp);
    }
    stokes::require(std::rename(tmp.c_str(), path) == 0, std::string("cannot rename to ") + path);
  });
}

// Merges the entries of a cache file into the process-wide cache. Lines
// that do not parse, name an unknown precision or variant, or whose shape
// (threads, targets per thread, tile) differs from this build's variant of
// that index are skipped; *n_loaded (may be NULL) counts the entries taken.
int stokes_tune_cache_load(const char* path, int* n_loaded) {
  return run([&] {
    stokes::require(path && *path, "null path");
    std::ifstream in(path);
    stokes::require((bool)in, std::string("cannot read ") + path);
    int taken = 0;
    std::string line;
    while (std::getline(in, line)) {
      double p, ln, lt, var, th, tpt, tile, cps, ms = 0.0;
      if (!stokes::json_number(line, "precision", p) || !stokes::json_number(line, "log2_sources", ln) ||
          !stokes::json_number(line, "log2_targets", lt) || !stokes::json_number(line, "variant", var) ||
          !stokes::json_number(line, "threads", th) || !stokes::json_number(line, "targets_per_thread", tpt) ||
          !stokes::json_number(line, "tile", tile) || !stokes::json_number(line, "ctas_per_sm", cps))
        continue;
      stokes::json_number(line, "ms", ms);
      const int prec = (int)p, v = (int)var, c = (int)cps;
      if (prec != STOKES_FP64 && prec != STOKES_FP32 && prec != STOKES_DF64) continue;
      if (ln < 0 || ln > 62 || lt < 0 || lt > 62) continue;
      if (!stokes::valid_shape(prec, v, c)) continue;
      stokes::PairVariant vars[stokes::kMaxVariants];
      stokes::variants_of(prec, vars);
      if (vars[v].threads != (int)th || vars[v].tpt != (int)tpt || vars[v].tile != (int)tile) continue;
      std::lock_guard<std::mutex> lk(stokes::g_cache_mu);
      stokes::g_cache[stokes::CacheKey(prec, (int)ln, (int)lt)] = stokes::CacheEntry{v, c, ms};
      ++taken;
    }
    if (n_loaded) *n_loaded = taken;
  });
}

}  // extern "C"
