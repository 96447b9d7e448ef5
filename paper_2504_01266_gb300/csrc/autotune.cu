// autotune.cu -- picks the launch configuration of the depthwise kernels per
// problem class by timing every candidate with CUDA events, and keeps the
// choices in memory and (optionally) in a JSON file.
//
// Candidates:
//   forward / input gradient: output rows per thread 8 (64 x 128 tiles) or
//                             4 (32 x 128 tiles: twice the CTAs, less halo reuse)
//                             x one tile per CTA or persistent CTAs x with or
//                             without an L2 prefetch of a later tile;
//   filter gradient (alone or fused): tiles per CTA = automatic, 2, 4, 8, 16
//                             (fewer partial sums vs. better load balance).
// Problem class: (op, dtype, K, border, floor(log2(N*C*H*W))).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "dw_launch.h"
#include "internal.h"

namespace giga {

static std::mutex g_mu;
static std::map<std::string, int> g_cache;
static int g_mode = -1;
static bool g_loaded = false;

static int env_mode() {
  const char* e = std::getenv("GIGA_AUTOTUNE");
  if (!e) return 1;
  if (!std::strcmp(e, "off") || !std::strcmp(e, "0")) return 0;
  if (!std::strcmp(e, "full") || !std::strcmp(e, "2")) return 2;
  return 1;
}

int tune_mode() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_mode < 0) g_mode = env_mode();
  return g_mode;
}

// Forward / input gradient: {8, 4} rows per thread x {one tile per CTA,
// persistent} x {no prefetch, L2 prefetch}; filter gradient: tiles per chunk {auto, 2, 4, 8, 16}; fused
// backward: the fused kernel with tiles per CTA {auto, 2, 4, 8, 16}, the
// two-pass split, or the persistent kernel with a tile ring (three stages where
// they fit, else two).
int tune_candidates(int op) {
  switch (op) {
    case TUNE_FWD:
    case TUNE_BWD_INPUT: return 8;
    case TUNE_BWD_FILTER: return 5;
    default: return 7;
  }
}


static int auto_tiles_per_cta(const DwArgs& a) {
  const int64_t tiles = a.N * a.C * (int64_t)((a.W + kTileW - 1) / kTileW) *
                        (int64_t)((a.H + 63) / 64);
  int64_t t = tiles / ((int64_t)sm_count() * 16);
  if (t < 1) t = 1;
  if (t > 16) t = 16;
  return (int)t;
}

// The persistent filter kernel runs one CTA per SM over chunks dealt round
// robin; a chunk ends with a reduction of the accumulators costing about a
// fifth of a tile.  Pick the chunk length (<= 16 tiles) minimising the
// busiest CTA's rounds x (tiles + 0.2).
static int auto_filter_tiles_per_chunk(const DwArgs& a) {
  const int64_t tpp = (int64_t)((a.W + kTileW - 1) / kTileW) * (int64_t)((a.H + 63) / 64);
  const int64_t planes = a.N * a.C;
  const int64_t G = sm_count();
  int best = 1;
  double best_cost = 1e300;
  for (int tpc = 16; tpc >= 1; tpc /= 2) {
    const int64_t chunks = planes * ((tpp + tpc - 1) / tpc);
    const double cost = (double)((chunks + G - 1) / G) * (tpc + 0.2);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = tpc;
    }
  }
  return best;
}

DwConfig tune_config(int op, int id, const DwArgs& a) {
  DwConfig c;
  c.rows_per_thread = 8;
  c.persistent = 0;
  c.prefetch = 0;
  c.split = 0;
  c.ring = 0;
  c.tiles_per_cta = op == TUNE_BWD_FILTER ? auto_filter_tiles_per_chunk(a) : auto_tiles_per_cta(a);
  static const int tpc[5] = {0, 2, 4, 8, 16};
  switch (op) {
    case TUNE_FWD:
    case TUNE_BWD_INPUT:
      c.rows_per_thread = (id & 1) ? 4 : 8;
      c.persistent = (id & 2) ? 1 : 0;
      c.prefetch = (id & 4) ? 1 : 0;
      break;
    case TUNE_BWD_FILTER:
      if (id >= 1 && id <= 4) c.tiles_per_cta = tpc[id];
      break;
    default:
      if (id >= 1 && id <= 4) c.tiles_per_cta = tpc[id];
      if (id == 5 || id == 6) {
        c.split = id == 5;
        c.ring = id == 6;
        c.tiles_per_cta = auto_filter_tiles_per_chunk(a);
      }
      break;
  }
  return c;
}

static std::string key_of(int op, const DwArgs& a) {
  const double n = (double)a.N * a.C * a.H * a.W;
  const int sc = n > 0 ? (int)std::floor(std::log2(n)) : 0;
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d", op, a.dtype, a.K, a.border, sc);
  return buf;
}

// ---- JSON persistence: {"giga_autotune": 1, "entries": {"key": id, ...}}
static bool parse_cache(const std::string& text, std::map<std::string, int>& out) {
  if (text.find("\"giga_autotune\"") == std::string::npos) return false;
  size_t p = text.find("\"entries\"");
  if (p == std::string::npos) return false;
  p = text.find('{', p);
  if (p == std::string::npos) return false;
  const size_t end = text.find('}', p);
  if (end == std::string::npos) return false;
  std::map<std::string, int> tmp;
  while (true) {
    size_t q0 = text.find('"', p);
    if (q0 == std::string::npos || q0 > end) break;
    size_t q1 = text.find('"', q0 + 1);
    if (q1 == std::string::npos || q1 > end) return false;
    std::string key = text.substr(q0 + 1, q1 - q0 - 1);
    size_t colon = text.find(':', q1);
    if (colon == std::string::npos || colon > end) return false;
    char* stop = nullptr;
    long v = std::strtol(text.c_str() + colon + 1, &stop, 10);
    if (stop == text.c_str() + colon + 1 || v < 0 || v > 64) return false;
    for (char ch : key)
      if (!(ch == ':' || ch == '-' || (ch >= '0' && ch <= '9'))) return false;
    tmp[key] = (int)v;
    p = (size_t)(stop - text.c_str());
  }
  out.swap(tmp);
  return true;
}

static bool load_file(const char* path) {
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  std::map<std::string, int> m;
  if (!parse_cache(ss.str(), m)) return false;  // a corrupt cache is ignored
  for (auto& kv : m) g_cache[kv.first] = kv.second;
  return true;
}

static bool save_file(const char* path) {
  std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\"giga_autotune\": 1, \"entries\": {";
    bool first = true;
    for (auto& kv : g_cache) {
      f << (first ? "" : ", ") << '"' << kv.first << "\": " << kv.second;
      first = false;
    }
    f << "}}\n";
  }
  return std::rename(tmp.c_str(), path) == 0;
}

static void ensure_loaded() {
  if (g_loaded) return;
  g_loaded = true;
  if (const char* p = std::getenv("GIGA_AUTOTUNE_CACHE")) load_file(p);
}

int tune_lookup(int op, const DwArgs& a) {
  std::lock_guard<std::mutex> lk(g_mu);
  ensure_loaded();
  auto it = g_cache.find(key_of(op, a));
  if (it == g_cache.end()) return -1;
  return it->second < tune_candidates(op) ? it->second : -1;
}

void tune_store(int op, const DwArgs& a, int id) {
  std::lock_guard<std::mutex> lk(g_mu);
  ensure_loaded();
  g_cache[key_of(op, a)] = id;
  if (const char* p = std::getenv("GIGA_AUTOTUNE_CACHE")) save_file(p);
}

// GIGA_LOG=1 (or any value but 0): each tuning decision is printed to
// standard error, one line per (op, problem class) with every candidate's time.
bool tune_log_enabled() {
  const char* e = std::getenv("GIGA_LOG");
  return e && *e && std::strcmp(e, "0") != 0;
}

static const char* op_name(int op) {
  switch (op) {
    case TUNE_FWD: return "forward";
    case TUNE_BWD_INPUT: return "input-gradient";
    case TUNE_BWD_FILTER: return "filter-gradient";
    default: return "fused-backward";
  }
}

giga_status_t tune_dw_op(int op, const DwArgs& a, cudaStream_t st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(GIGA_ERR_CUDA, "event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(GIGA_ERR_CUDA, "event create");
  }
  int best = 0;
  float best_ms = 1e30f;
  std::string times;
  giga_status_t status = GIGA_OK;
  for (int id = 0; id < tune_candidates(op) && status == GIGA_OK; ++id) {
    const DwConfig cfg = tune_config(op, id, a);
    status = run_dw_op(op, a, cfg, st);  // warm-up
    if (status != GIGA_OK) break;
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 3 && status == GIGA_OK; ++rep) status = run_dw_op(op, a, cfg, st);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      status = cuda_fail(e, "autotune timing");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    char buf[48];
    std::snprintf(buf, sizeof(buf), "%s%d:%.3f", id ? " " : "", id, ms / 3.f);
    times += buf;
    if (ms < best_ms) {
      best_ms = ms;
      best = id;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status == GIGA_OK) {
    tune_store(op, a, best);
    if (tune_log_enabled())
      std::fprintf(stderr,
                   "giga autotune: %s %s K=%d %s N*C*H*W=%lld (class %s) -> candidate %d "
                   "(ms per call: %s)\n",
                   op_name(op), a.dtype ? "bf16" : "f32", a.K, a.border ? "clamp" : "zero",
                   (long long)(a.N * a.C * a.H * a.W), key_of(op, a).c_str(), best,
                   times.c_str());
  }
  return status;
}

}  // namespace giga

using namespace giga;

extern "C" {

giga_status_t giga_autotune_set_mode(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 2) return fail(GIGA_ERR_INVALID_ARG, "autotune mode must be 0, 1 or 2");
  std::lock_guard<std::mutex> lk(g_mu);
  g_mode = mode;
  return GIGA_OK;
}

int32_t giga_autotune_get_mode(void) { return tune_mode(); }

giga_status_t giga_autotune_save(const char* path) {
  clear_error();
  if (!path) return fail(GIGA_ERR_INVALID_ARG, "path is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  return save_file(path) ? GIGA_OK : fail(GIGA_ERR_INVALID_ARG, "cannot write autotune cache");
}

giga_status_t giga_autotune_load(const char* path) {
  clear_error();
  if (!path) return fail(GIGA_ERR_INVALID_ARG, "path is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  g_loaded = true;
  return load_file(path) ? GIGA_OK
                         : fail(GIGA_ERR_INVALID_ARG, "autotune cache missing or corrupt (ignored)");
}

void giga_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}

}  // extern "C"
