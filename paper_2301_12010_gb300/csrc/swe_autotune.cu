// swe_autotune.cu -- tile-shape autotuner: times every compiled tile shape
// on a synthetic scenario of the requested size (single-scenario path or a
// batch of the given grids) and keeps the winner in a JSON cache keyed by
// (GPU name, precision, mode, size bucket).  swe_create / swe_batch_create
// consult the cache when params->tile == 0.
#include <sys/stat.h>

#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "swe_launch.h"
#include "swe_trace.h"

namespace {

std::mutex g_cache_lock;

// mkdir -p of the directories above a file path
void make_parents(const std::string &path) {
  for (size_t k = 1; k < path.size(); ++k)
    if (path[k] == '/') {
      const std::string part = path.substr(0, k);
      if (mkdir(part.c_str(), 0755) != 0 && errno != EEXIST) return;
    }
}

std::string cache_path() {
  const char *p = std::getenv("SWE_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char *home = std::getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/swe_gb300_autotune.json";
}

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp pr;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return "unknown";
  }
  return pr.name;
}

int bucket_of(double cells) { return cells > 1.0 ? (int)std::floor(std::log2(cells)) : 0; }

std::string key_of(int precision, int mode, int bucket) {
  char b[256];
  std::snprintf(b, sizeof b, "%s|%s|%s|%d", gpu_name().c_str(), precision == SWE_F64 ? "f64" : "f32",
                mode == 1 ? "batch" : "single", bucket);
  return b;
}

// Cache file: a JSON object, one entry per line:
//   "GPU|prec|mode|bucket": {"tile": k, "ms": [..]},
std::map<std::string, std::string> read_cache() {
  std::map<std::string, std::string> m;
  FILE *f = std::fopen(cache_path().c_str(), "r");
  if (!f) return m;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    const char *q1 = std::strchr(line, '"');
    if (!q1) continue;
    const char *q2 = std::strchr(q1 + 1, '"');
    if (!q2) continue;
    const char *colon = std::strchr(q2, ':');
    if (!colon) continue;
    std::string val(colon + 1);
    while (!val.empty() && (val.back() == '\n' || val.back() == ',' || val.back() == ' ')) val.pop_back();
    m[std::string(q1 + 1, q2)] = val;
  }
  std::fclose(f);
  return m;
}

void write_cache(const std::map<std::string, std::string> &m) {
  const std::string path = cache_path();
  make_parents(path);
  const std::string tmp = path + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t n = 0;
  for (auto &kv : m) std::fprintf(f, " \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++n < m.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

int tile_from(const std::string &val) {
  const char *t = std::strstr(val.c_str(), "\"tile\"");
  if (!t) return 0;
  t = std::strchr(t, ':');
  return t ? std::atoi(t + 1) : 0;
}

// Synthetic tuning scenario: still water over a sloping bed with a smooth
// hump of surface elevation (moving water, no dry cells).
void synthetic(int nx, int ny, std::vector<double> &b, std::vector<double> &h, std::vector<double> &z) {
  b.resize((size_t)nx * ny);
  h.resize(b.size());
  z.assign(b.size(), 0.0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i + 0.5) / nx, y = (j + 0.5) / ny;
      const size_t o = (size_t)j * nx + i;
      b[o] = -20.0 + 10.0 * x + std::sin(20.0 * x) * std::cos(17.0 * y);
      const double r2 = (x - 0.3) * (x - 0.3) + (y - 0.5) * (y - 0.5);
      h[o] = -b[o] + 0.5 * std::exp(-r2 / 0.01);
    }
}

}  // namespace

extern "C" {

int swe_autotune(const swe_grid *grids, int32_t ngrids, int32_t precision, int32_t mode, int32_t steps,
                 int32_t *best_tile, double *ms) {
  const swe::TraceRange trace("swe_autotune");
  if (!grids || ngrids < 1 || (mode != 0 && mode != 1) || steps < 1 || !best_tile) return SWE_EINVAL;
  if (mode == 1 && precision != SWE_F32) return SWE_EINVAL;
  for (int g = 0; g < ngrids; ++g)
    if (grids[g].nx < 3 || grids[g].ny < 3) return SWE_EINVAL;
  const int nshapes = swe_tile_count();
  std::vector<double> t(nshapes + 1, INFINITY);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SWE_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double cells = 0.0;
  for (int g = 0; g < ngrids; ++g) cells += (double)grids[g].nx * grids[g].ny;
  int rc = SWE_OK;
  for (int k = 1; k <= nshapes && rc == SWE_OK; ++k) {
    swe_params p;
    swe_params_default(&p);
    p.precision = precision;
    p.tile = k;
    p.stream = st;
    float msk = 0.f;
    if (mode == 0) {
      std::vector<double> b, h, z;
      synthetic(grids[0].nx, grids[0].ny, b, h, z);
      swe_handle *s = nullptr;
      int r = swe_create(&grids[0], 1.0, 1.0, b.data(), &p, &s);
      if (r == SWE_EINVAL) continue;  // shape does not fit this precision
      if (r != SWE_OK) { rc = r; break; }
      r = swe_set_state(s, h.data(), z.data(), z.data());
      if (r == SWE_OK) r = swe_step(s, 2, 0.4);
      if (r == SWE_OK) r = swe_sync(s);
      if (r == SWE_OK) {
        cudaEventRecord(e0, st);
        r = swe_step(s, steps, 0.4);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&msk, e0, e1);
      }
      swe_destroy(s);
      if (r != SWE_OK) { rc = r; break; }
    } else {
      swe_batch *bt = nullptr;
      size_t need = 0;
      for (int g = 0; g < ngrids; ++g) need += swe_batch_slot_bytes(&grids[g]);
      int r = swe_batch_create(ngrids, need, &p, &bt);
      if (r != SWE_OK) { rc = r; break; }
      for (int g = 0; g < ngrids && r == SWE_OK; ++g) {
        std::vector<double> b, h, z;
        synthetic(grids[g].nx, grids[g].ny, b, h, z);
        int32_t slot;
        r = swe_batch_admit(bt, &grids[g], 1.0, 1.0, b.data(), h.data(), z.data(), z.data(), 1e30, &slot);
      }
      if (r == SWE_OK) r = swe_batch_run(bt, 1, 0.4);
      if (r == SWE_OK) r = swe_batch_status(bt);
      if (r == SWE_OK) {
        cudaEventRecord(e0, st);
        r = swe_batch_run(bt, steps, 0.4);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&msk, e0, e1);
        if (r == SWE_OK) r = swe_batch_status(bt);
      }
      swe_batch_destroy(bt);
      if (r != SWE_OK) { rc = r; break; }
    }
    t[k] = msk / steps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc != SWE_OK) return rc;
  int best = 1;
  for (int k = 1; k <= nshapes; ++k)
    if (t[k] < t[best]) best = k;
  *best_tile = best;
  if (ms)
    for (int k = 1; k <= nshapes; ++k) ms[k - 1] = std::isfinite(t[k]) ? t[k] : -1.0;
  char val[512];
  int n = std::snprintf(val, sizeof val, "{\"tile\": %d, \"ms_per_step\": [", best);
  for (int k = 1; k <= nshapes; ++k)
    n += std::snprintf(val + n, sizeof val - n, "%s%.6g", k > 1 ? ", " : "", std::isfinite(t[k]) ? t[k] : -1.0);
  std::snprintf(val + n, sizeof val - n, "]}");
  std::lock_guard<std::mutex> guard(g_cache_lock);
  auto m = read_cache();
  m[key_of(precision, mode, mode == 1 ? -1 : bucket_of(cells))] = val;
  write_cache(m);
  return SWE_OK;
}

int swe_autotune_lookup(int32_t precision, int32_t mode, double cells) {
  std::lock_guard<std::mutex> guard(g_cache_lock);
  auto m = read_cache();
  auto it = m.find(key_of(precision, mode, mode == 1 ? -1 : bucket_of(cells)));
  if (it == m.end()) return 0;
  const int t = tile_from(it->second);
  return (t >= 1 && t <= swe_tile_count()) ? t : 0;
}

}  // extern "C"
