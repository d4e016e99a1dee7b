// Launch-configuration autotuner.
//
// Some launch parameters have no best value across meshes, trial widths and
// numbers of Bloch vectors in flight (how many partial blocks a Gram reduction
// uses, which Gram kernel runs, how wide the block-update grid is).  The first
// time a kernel meets a new shape, pick() runs each candidate configuration on
// the real data (once to warm up, then twice timed with CUDA events on the
// launching stream) and keeps the fastest; the choice is remembered for the
// process and written to a small JSON file (PBS_TUNE_CACHE, default
// $HOME/.cache/pbs_tune.json; PBS_TUNE=0 switches tuning off and takes the first
// candidate), so later processes on the same device start from it.  Candidates
// must be idempotent: each run overwrites its outputs from unchanged inputs.
// PBS_TUNE_FORCE="prefix=i,prefix=j,..." makes every key that begins with a listed
// prefix take candidate i (where it exists) without timing, so that tests can run
// each candidate.
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include <sys/stat.h>

#include "internal.h"

namespace pbs {
namespace {

struct TuneCache {
  std::mutex mu;
  std::map<std::string, int> choice;
  bool loaded = false;
  std::string path;
};

TuneCache& cache() {
  static TuneCache c;
  return c;
}

bool tuning_on() {
  static const bool on = [] {
    const char* v = std::getenv("PBS_TUNE");
    return !(v && std::strcmp(v, "0") == 0);
  }();
  return on;
}

// PBS_TUNE_FORCE entries (prefix, candidate), read once
const std::vector<std::pair<std::string, int>>& forced() {
  static const std::vector<std::pair<std::string, int>> f = [] {
    std::vector<std::pair<std::string, int>> v;
    const char* e = std::getenv("PBS_TUNE_FORCE");
    if (!e) return v;
    std::stringstream ss(e);
    std::string item;
    while (std::getline(ss, item, ',')) {
      const size_t eq = item.rfind('=');
      if (eq == std::string::npos || eq == 0) continue;
      v.emplace_back(item.substr(0, eq), std::atoi(item.c_str() + eq + 1));
    }
    return v;
  }();
  return f;
}

std::string cache_path() {
  if (const char* p = std::getenv("PBS_TUNE_CACHE")) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/pbs_tune.json";
}

// {"key": index, ...}: keys hold no quotes or backslashes
void load(TuneCache& c) {
  c.loaded = true;
  c.path = cache_path();
  std::ifstream f(c.path);
  if (!f) return;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t pos = 0;
  for (;;) {
    const size_t k0 = s.find('"', pos);
    if (k0 == std::string::npos) break;
    const size_t k1 = s.find('"', k0 + 1);
    if (k1 == std::string::npos) break;
    const size_t colon = s.find(':', k1);
    if (colon == std::string::npos) break;
    const int v = std::atoi(s.c_str() + colon + 1);
    c.choice[s.substr(k0 + 1, k1 - k0 - 1)] = v;
    pos = colon + 1;
  }
}

void save(const TuneCache& c) {
  const size_t slash = c.path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = c.path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)  // each missing directory of the path (errors ignored)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = c.path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;  // an unwritable cache only costs re-tuning in the next process
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : c.choice)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < c.choice.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), c.path.c_str());
}

}  // namespace

std::string device_tag() {
  static std::mutex mu;
  static std::map<int, std::string> tags;  // per device: the properties query is slow
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return "dev";
  std::lock_guard<std::mutex> lk(mu);
  auto it = tags.find(dev);
  if (it != tags.end()) return it->second;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "dev";
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == '"' || ch == '\\' || ch == ' ') ch = '_';
  name += "_sm" + std::to_string(prop.multiProcessorCount);
  tags[dev] = name;
  return name;
}

int tune_pick(const std::string& key, int ncand, const std::function<void(int)>& run, cudaStream_t s) {
  if (ncand <= 1) return 0;
  for (const auto& f : forced())
    if (key.compare(0, f.first.size(), f.first) == 0 && f.second >= 0 && f.second < ncand) return f.second;
  if (!tuning_on()) return 0;
  TuneCache& c = cache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    if (!c.loaded) load(c);
    auto it = c.choice.find(key);
    if (it != c.choice.end() && it->second >= 0 && it->second < ncand) return it->second;
  }
  // time every candidate on this stream (outside the lock: other threads tune other keys)
  cudaEvent_t e0, e1;
  PBS_CUDA(cudaEventCreate(&e0));
  PBS_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.0f;
  try {
    for (int cand = 0; cand < ncand; ++cand) {
      run(cand);  // warm-up (lazy set-up, caches)
      PBS_CUDA(cudaEventRecord(e0, s));
      run(cand);
      run(cand);
      PBS_CUDA(cudaEventRecord(e1, s));
      PBS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      PBS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (verbose_enabled()) std::fprintf(stderr, "[pbs] tune %s candidate %d: %.3f ms per run\n", key.c_str(), cand, ms / 2);
      if (cand == 0 || ms < best_ms) {
        best = cand;
        best_ms = ms;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (verbose_enabled()) std::fprintf(stderr, "[pbs] tuned %s -> %d (%.3f ms per run)\n", key.c_str(), best, best_ms / 2);
  std::lock_guard<std::mutex> lk(c.mu);
  c.choice[key] = best;
  save(c);
  return best;
}

}  // namespace pbs
