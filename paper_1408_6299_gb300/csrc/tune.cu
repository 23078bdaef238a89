// tune.cu -- the persistent store of the autotuner's choices (the column-pass
// variant and the row-block size of the real-to-complex pass per shape,
// precision and stack size; see fused_launch.cuh). Choices are kept per
// process and in a JSON file, one object of "key": choice pairs, so later
// processes reuse them without timing trials. The file is
// $REG_TUNE_CACHE when that is set (an empty value disables the file), else
// tune_cache.json beside the library. Keys begin with the device name and
// its multiprocessor count, so one file can serve several GPU types.
#include <dlfcn.h>
#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace reg {
namespace {

std::mutex g_mu;
bool g_loaded = false;
std::map<std::string, int> g_choice;

std::string cache_path() {
  const char* env = getenv("REG_TUNE_CACHE");
  if (env) return std::string(env);
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&tune_lookup), &info) && info.dli_fname) {
    std::string p(info.dli_fname);
    const size_t slash = p.rfind('/');
    return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/tune_cache.json";
  }
  return "";
}

// the file holds one flat JSON object of string keys and integer values
void load_locked() {
  g_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  size_t i = 0;
  for (;;) {
    const size_t a = text.find('"', i);
    if (a == std::string::npos) break;
    const size_t b = text.find('"', a + 1);
    if (b == std::string::npos) break;
    const size_t colon = text.find(':', b);
    if (colon == std::string::npos) break;
    char* end = nullptr;
    const long v = strtol(text.c_str() + colon + 1, &end, 10);
    if (end == text.c_str() + colon + 1) break;
    g_choice[text.substr(a + 1, b - a - 1)] = (int)v;
    i = (size_t)(end - text.c_str());
  }
}

void save_locked() {
  const std::string path = cache_path();
  if (path.empty()) return;
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fputs("{\n", f);
  size_t k = 0;
  for (const auto& e : g_choice)
    fprintf(f, "  \"%s\": %d%s\n", e.first.c_str(), e.second, ++k < g_choice.size() ? "," : "");
  fputs("}\n", f);
  const bool ok = fclose(f) == 0;
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

}  // namespace

std::string tune_device_tag() {
  int dev = 0, sms = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return "unknown";
  }
  sms = p.multiProcessorCount;
  return std::string(p.name) + "/" + std::to_string(sms);
}

int tune_lookup(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_locked();
  auto it = g_choice.find(key);
  return it == g_choice.end() ? -1 : it->second;
}

void tune_store(const std::string& key, int choice) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_locked();
  g_choice[key] = choice;
  save_locked();
}

}  // namespace reg
