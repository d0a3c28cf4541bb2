// Persisted launch shapes: the shapes hj_autotune (or hj_set_launch_shape) stored
// on a problem, written to and read from a text file so that a later process
// on the same kind of GPU skips the tuning.
//
// One line per stored shape, fields separated by '|':
//   <GPU name>|<family>|<d>|<precision>|<N>|<warps per point>|<nodes per lane>
// (warps per point 0: half a warp).  Saving merges into the file: a line with
// the same (GPU name, family, d, precision, N) is replaced, every other line is
// kept.  Loading applies the lines that match the current device's name and the
// problem's (family, d), through the checks of hj_set_launch_shape; lines that
// do not parse or do not pass are skipped.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "hj_internal.cuh"
#include "hjpdhg.h"
#include "problem.cuh"

namespace {

struct Entry {
  std::string gpu;
  int family = 0, d = 0, precision = 0, N = 0, warps = 0, npl = 0;
};

bool device_name(int dev, std::string* out) {
  cudaDeviceProp pr{};
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return false;
  *out = pr.name;
  for (char& ch : *out)
    if (ch == '|' || ch == '\n' || ch == '\r') ch = ' ';
  return true;
}

bool parse(const std::string& line, Entry* e) {
  std::vector<std::string> f;
  size_t a = 0;
  for (;;) {
    const size_t b = line.find('|', a);
    f.push_back(line.substr(a, b == std::string::npos ? std::string::npos : b - a));
    if (b == std::string::npos) break;
    a = b + 1;
  }
  if (f.size() != 7 || f[0].empty()) return false;
  int v[6];
  for (int i = 0; i < 6; ++i) {
    char* end = nullptr;
    const long x = std::strtol(f[i + 1].c_str(), &end, 10);
    if (end == f[i + 1].c_str() || *end != '\0' || x < -1000000 || x > 1000000) return false;
    v[i] = (int)x;
  }
  e->gpu = f[0];
  e->family = v[0]; e->d = v[1]; e->precision = v[2]; e->N = v[3]; e->warps = v[4]; e->npl = v[5];
  return true;
}

std::vector<std::string> read_lines(const char* path) {
  std::vector<std::string> lines;
  FILE* fp = std::fopen(path, "r");
  if (fp == nullptr) return lines;
  char buf[512];
  std::string cur;
  while (std::fgets(buf, sizeof(buf), fp) != nullptr) {
    cur += buf;
    if (!cur.empty() && cur.back() == '\n') {
      cur.pop_back();
      if (!cur.empty() && cur.back() == '\r') cur.pop_back();
      lines.push_back(cur);
      cur.clear();
    }
  }
  if (!cur.empty()) lines.push_back(cur);
  std::fclose(fp);
  return lines;
}

}  // namespace

extern "C" {

hj_status hj_shapes_save(hj_problem prob, const char* path) {
  if (prob == nullptr || path == nullptr) return HJ_ERR_INVALID_ARG;
  std::string gpu;
  if (!device_name(prob->device, &gpu)) return HJ_ERR_CUDA;
  std::map<std::pair<int, int>, hj::WarpConfig> shapes;
  {
    std::lock_guard<std::mutex> g(prob->mu);
    shapes = prob->shapes;
  }
  // the file's other lines, minus the ones this save replaces
  std::vector<std::string> keep;
  for (const std::string& line : read_lines(path)) {
    Entry e;
    const bool mine = parse(line, &e) && e.gpu == gpu && e.family == prob->family &&
                      e.d == prob->d && shapes.count({e.precision, e.N}) != 0;
    if (!mine && !line.empty()) keep.push_back(line);
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* fp = std::fopen(tmp.c_str(), "w");
  if (fp == nullptr) return HJ_ERR_INVALID_ARG;
  bool ok = true;
  for (const std::string& line : keep) ok = ok && std::fprintf(fp, "%s\n", line.c_str()) > 0;
  for (const auto& kv : shapes) {
    const hj::WarpConfig& c = kv.second;
    ok = ok && std::fprintf(fp, "%s|%d|%d|%d|%d|%d|%d\n", gpu.c_str(), prob->family, prob->d,
                            kv.first.first, kv.first.second, c.half ? 0 : c.G, c.NPL) > 0;
  }
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return HJ_ERR_INVALID_ARG;
  }
  return HJ_OK;
}

hj_status hj_shapes_load(hj_problem prob, const char* path, int32_t* n_loaded) {
  if (prob == nullptr || path == nullptr) return HJ_ERR_INVALID_ARG;
  if (n_loaded != nullptr) *n_loaded = 0;
  std::string gpu;
  if (!device_name(prob->device, &gpu)) return HJ_ERR_CUDA;
  int32_t n = 0;
  for (const std::string& line : read_lines(path)) {
    Entry e;
    if (!parse(line, &e) || e.gpu != gpu || e.family != prob->family || e.d != prob->d) continue;
    if (hj_set_launch_shape(prob, e.precision, e.N, e.warps, e.npl) == HJ_OK) ++n;
  }
  if (n_loaded != nullptr) *n_loaded = n;
  return HJ_OK;
}

}  // extern "C"
