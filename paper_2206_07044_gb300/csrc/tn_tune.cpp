// Per-device table of autotuned launch shapes (tn_tune.h).
#include "tn_tune.h"

#include <cuda_runtime.h>

#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>

namespace tnk {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // device, kernel, m, n, k, batch

std::mutex g_mu;
std::map<Key, int> g_table;

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  return dev;
}

// "name|SMs" of the current device: a cache is applied only to the same model.
std::string device_tag() {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, current_device()) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string name = p.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "|" + std::to_string(p.multiProcessorCount);
}

}  // namespace

int tune_get(int kernel, int m, int n, int k, int batch) {
  const Key key{current_device(), kernel, m, n, k, batch};
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(key);
  return it == g_table.end() ? 0 : it->second;
}

void tune_set(int kernel, int m, int n, int k, int batch, int value) {
  const Key key{current_device(), kernel, m, n, k, batch};
  std::lock_guard<std::mutex> lk(g_mu);
  if (value == 0)
    g_table.erase(key);
  else
    g_table[key] = value;
}

int tune_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  int c = 0;
  for (const auto& e : g_table) c += std::get<0>(e.first) == dev;
  return c;
}

std::vector<std::vector<int>> tune_entries() {
  const int dev = current_device();
  std::vector<std::vector<int>> out;
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto& e : g_table)
    if (std::get<0>(e.first) == dev)
      out.push_back({std::get<1>(e.first), std::get<2>(e.first), std::get<3>(e.first), std::get<4>(e.first),
                     std::get<5>(e.first), e.second});
  return out;
}

std::string tune_save(const std::string& path) {
  const std::string tag = device_tag();
  std::ofstream f(path, std::ios::trunc);
  if (!f) return "cannot write " + path;
  f << "tntune 1 " << tag << "\n";
  for (const auto& r : tune_entries())
    f << r[0] << " " << r[1] << " " << r[2] << " " << r[3] << " " << r[4] << " " << r[5] << "\n";
  return f ? "" : "write failed: " + path;
}

std::string tune_load(const std::string& path) {
  std::ifstream f(path);
  if (!f) return "";  // no cache yet: nothing to load
  std::string line;
  if (!std::getline(f, line)) return "";
  std::istringstream hs(line);
  std::string magic, ver, tag;
  hs >> magic >> ver >> tag;
  if (magic != "tntune" || ver != "1") return "not a tuning cache: " + path;
  if (tag != device_tag()) return "";  // taken on another GPU model: ignored
  int kernel, m, n, k, batch, value;
  while (f >> kernel >> m >> n >> k >> batch >> value) {
    if (kernel < TK_QR || kernel > TK_GEMMTC || value <= 0) return "malformed tuning cache: " + path;
    tune_set(kernel, m, n, k, batch, value);
  }
  return "";
}

}  // namespace tnk
