// Launch-shape autotuner.  Kernels with several launch shapes (lanes per CSR row, stencil
// tile and plane counts, multivector block shapes) register the shapes as numbered
// variants.  autotune() times every variant of one launch with CUDA events on the
// caller's stream and caches the fastest under (kernel, shape key); launchers then ask
// tuned_variant() for the cached choice and fall back to a fixed default when the key
// has not been tuned.  Choices are per process (optionally persisted to the file named
// by FEM_AUTOTUNE_CACHE); FEM_AUTOTUNE=0 disables timing, so every launch takes its
// default.  A tuned choice changes only the order of floating-point sums, never the
// arithmetic performed.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace fem {

namespace {

struct TuneEntry {
  std::string kernel;
  int64_t a = 0, b = 0;
  int c = 0;
  int pick = 0;
  std::string source;                 // "timed", "file"
  std::vector<std::string> names;     // variant names
  std::vector<double> us;             // measured microseconds per launch (timed only)
};

struct Tuner {
  std::mutex mu;
  std::vector<std::pair<std::string, int>> pins;   // kernel -> variant for every shape
  std::unordered_map<uint64_t, int> pick;   // fast lookup
  std::vector<TuneEntry> entries;           // report, in tuning order
  bool loaded = false;
  int enabled = -1;
};

Tuner& tuner() {
  static Tuner t;
  return t;
}

uint64_t key_of(const char* kernel, int64_t a, int64_t b, int c) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the name, then mixed with the shape
  for (const char* p = kernel; *p; p++) {
    h ^= (unsigned char)*p;
    h *= 1099511628211ull;
  }
  auto mix = [&](uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  };
  mix((uint64_t)a);
  mix((uint64_t)b);
  mix((uint64_t)(uint32_t)c);
  return h;
}

bool tuning_enabled(Tuner& t) {
  if (t.enabled < 0) {
    const char* e = std::getenv("FEM_AUTOTUNE");
    t.enabled = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
  }
  return t.enabled == 1;
}

const char* cache_path() {
  const char* p = std::getenv("FEM_AUTOTUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

// Cache file: one line per choice, "kernel a b c pick".
void load_cache(Tuner& t) {
  if (t.loaded) return;
  t.loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char name[64];
  long long a, b;
  int c, pick;
  while (std::fscanf(f, "%63s %lld %lld %d %d", name, &a, &b, &c, &pick) == 5) {
    const uint64_t k = key_of(name, a, b, c);
    if (t.pick.count(k)) continue;
    t.pick[k] = pick;
    TuneEntry e;
    e.kernel = name;
    e.a = a;
    e.b = b;
    e.c = c;
    e.pick = pick;
    e.source = "file";
    t.entries.push_back(e);
  }
  std::fclose(f);
}

void append_cache(const TuneEntry& e) {
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %lld %lld %d %d\n", e.kernel.c_str(), (long long)e.a, (long long)e.b, e.c,
               e.pick);
  std::fclose(f);
}

int pinned(const Tuner& t, const char* kernel, int nvariants) {
  for (const auto& p : t.pins)
    if (p.first == kernel && p.second >= 0 && p.second < nvariants) return p.second;
  return -1;
}

}  // namespace

int tuned_variant(const char* kernel, int64_t a, int64_t b, int c, int def, int nvariants) {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> g(t.mu);
  if (!t.pins.empty()) {
    const int p = pinned(t, kernel, nvariants);
    if (p >= 0) return p;
  }
  load_cache(t);
  auto it = t.pick.find(key_of(kernel, a, b, c));
  if (it == t.pick.end() || it->second < 0 || it->second >= nvariants) return def;
  return it->second;
}

int autotune(const char* kernel, int64_t a, int64_t b, int c, int nvariants,
             const char* const* names, int def, cudaStream_t st,
             const std::function<void(int)>& run) {
  Tuner& t = tuner();
  {
    std::lock_guard<std::mutex> g(t.mu);
    const int p = pinned(t, kernel, nvariants);
    if (p >= 0) return p;
    load_cache(t);
    auto it = t.pick.find(key_of(kernel, a, b, c));
    if (it != t.pick.end() && it->second >= 0 && it->second < nvariants) return it->second;
    if (!tuning_enabled(t)) return def;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FEM_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return def;
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  std::vector<double> us(nvariants, 0.0);
  try {
    for (int v = 0; v < nvariants; v++) {
      run(v);   // warm-up (and first touch of the variant's code)
      FEM_CUDA(cudaEventRecord(e0, st));
      run(v);
      FEM_CUDA(cudaEventRecord(e1, st));
      FEM_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      FEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      // short launches: repeat to get above the timer's resolution
      int reps = ms < 0.05f ? 20 : (ms < 0.5f ? 5 : 2);
      FEM_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; r++) run(v);
      FEM_CUDA(cudaEventRecord(e1, st));
      FEM_CUDA(cudaEventSynchronize(e1));
      FEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      us[v] = 1e3 * (double)ms / reps;
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // fastest; the default keeps its place unless another variant beats it by 3%
  int best = 0;
  for (int v = 1; v < nvariants; v++)
    if (us[v] < us[best]) best = v;
  if (us[best] >= 0.97 * us[def]) best = def;
  TuneEntry e;
  e.kernel = kernel;
  e.a = a;
  e.b = b;
  e.c = c;
  e.pick = best;
  e.source = "timed";
  for (int v = 0; v < nvariants; v++) e.names.push_back(names ? names[v] : std::to_string(v));
  e.us = us;
  {
    std::lock_guard<std::mutex> g(t.mu);
    const uint64_t k = key_of(kernel, a, b, c);
    if (!t.pick.count(k)) {
      t.pick[k] = best;
      t.entries.push_back(e);
      append_cache(e);
    }
    return t.pick[k];
  }
}

std::string autotune_report() {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> g(t.mu);
  load_cache(t);
  std::ostringstream o;
  o << "{\"enabled\": " << (tuning_enabled(t) ? "true" : "false") << ", \"pins\": {";
  for (size_t i = 0; i < t.pins.size(); i++)
    o << (i ? ", " : "") << "\"" << t.pins[i].first << "\": " << t.pins[i].second;
  o << "}, \"entries\": [";
  for (size_t i = 0; i < t.entries.size(); i++) {
    const TuneEntry& e = t.entries[i];
    if (i) o << ", ";
    o << "{\"kernel\": \"" << e.kernel << "\", \"a\": " << e.a << ", \"b\": " << e.b
      << ", \"c\": " << e.c << ", \"source\": \"" << e.source << "\", \"pick\": " << e.pick;
    if (!e.names.empty()) o << ", \"pick_name\": \"" << e.names[e.pick] << "\"";
    o << ", \"variants\": [";
    for (size_t v = 0; v < e.names.size(); v++) {
      if (v) o << ", ";
      char buf[64];
      std::snprintf(buf, sizeof buf, "%.3f", e.us[v]);
      o << "{\"name\": \"" << e.names[v] << "\", \"us\": " << buf << "}";
    }
    o << "]}";
  }
  o << "]}";
  return o.str();
}

void autotune_pin(const char* kernel, int variant) {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> g(t.mu);
  for (auto it = t.pins.begin(); it != t.pins.end(); ++it)
    if (it->first == kernel) {
      t.pins.erase(it);
      break;
    }
  if (variant >= 0) t.pins.emplace_back(kernel, variant);
}

void autotune_clear() {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> g(t.mu);
  t.pick.clear();
  t.entries.clear();
  t.pins.clear();
  t.loaded = true;   // a cleared table does not re-read the file
}

}  // namespace fem
