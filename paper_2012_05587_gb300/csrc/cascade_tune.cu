// Persistent choices of the batch autotuner: size-class keys and the cache
// file that maps each key to the fastest launch variant of the batched
// particle kernel measured for it.  Host code only (no kernels).
//
// Key: precision, ceil(log2(largest grid)), nearest log2 of the particles,
// ceil(log2(members)) -- batches in one class share their launch shape.
// File: one line per key, "<key>\t<shape> <stage> <prefetch> <member_cost>\t<ns per unit>",
// rewritten whole (to a temporary file, then renamed) on every store, so a
// reader never sees a partial file.  Entries are also kept in memory, so a
// process that cannot write the file still reuses its own measurements.
#include <errno.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cascade_internal.h"

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::map<std::string, cascade_batch_variant>> g_mem;  // path -> key -> variant

int ceil_log2(double v) {
  if (!(v > 1.0)) return 0;
  return (int)ceil(log2(v) - 1e-12);
}

bool parse_line(const char* line, std::string* key, cascade_batch_variant* v) {
  const char* tab = strchr(line, '\t');
  if (!tab || tab == line) return false;
  key->assign(line, (size_t)(tab - line));
  int a, b, c, d;
  if (sscanf(tab + 1, "%d %d %d %d", &a, &b, &c, &d) != 4) return false;
  v->shape = a;
  v->stage = b;
  v->prefetch = c;
  v->member_cost = d;
  return true;
}

// Creates the directories above a file path (mkdir -p of its dirname).
void make_parent_dirs(const std::string& path) {
  for (size_t i = 1; i < path.size(); ++i) {
    if (path[i] != '/') continue;
    const std::string dir = path.substr(0, i);
    if (mkdir(dir.c_str(), 0755) != 0 && errno != EEXIST) return;
  }
}

}  // namespace

extern "C" {

int cascade_tune_key(int32_t precision, int32_t max_nx, int64_t particles, int32_t members, char* key_out,
                     int32_t key_len) {
  cpic::set_error_message("");
  if (!key_out || key_len < 64 || max_nx < 1 || particles < 0 || members < 1 ||
      (precision != CASCADE_FP64 && precision != CASCADE_FP32_MIXED && precision != CASCADE_FP32_MIXED_FINE))
    return CASCADE_ERR_INVALID_ARG;
  const int pc = particles > 0 ? (int)lround(log2((double)particles)) : 0;
  snprintf(key_out, (size_t)key_len, "prec%d-nx2^%d-np2^%d-m2^%d", precision, ceil_log2(max_nx), pc,
           ceil_log2(members));
  return CASCADE_OK;
}

int cascade_tune_cache_lookup(const char* path, const char* key, cascade_batch_variant* out, int32_t* found) {
  cpic::set_error_message("");
  if (!key || !out || !found) return CASCADE_ERR_INVALID_ARG;
  *found = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const std::string p = path ? path : "";
  auto it = g_mem.find(p);
  if (it != g_mem.end()) {
    auto jt = it->second.find(key);
    if (jt != it->second.end()) {
      *out = jt->second;
      *found = 1;
      return CASCADE_OK;
    }
  }
  if (p.empty()) return CASCADE_OK;
  FILE* f = fopen(p.c_str(), "r");
  if (!f) return CASCADE_OK;  // no file yet: nothing cached
  char line[512];
  std::string k;
  cascade_batch_variant v{};
  while (fgets(line, sizeof(line), f)) {
    if (parse_line(line, &k, &v) && k == key) {  // the last line for a key wins
      *out = v;
      *found = 1;
    }
  }
  fclose(f);
  if (*found) g_mem[p][key] = *out;
  return CASCADE_OK;
}

int cascade_tune_cache_store(const char* path, const char* key, const cascade_batch_variant* v,
                             double ns_per_unit) {
  cpic::set_error_message("");
  if (!key || !v || !*key || strchr(key, '\t') || strchr(key, '\n')) return CASCADE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const std::string p = path ? path : "";
  g_mem[p][key] = *v;
  if (p.empty()) return CASCADE_OK;
  // keep the other keys' lines (last one per key), replace this key's
  std::vector<std::string> order;
  std::map<std::string, std::string> lines;
  FILE* f = fopen(p.c_str(), "r");
  if (f) {
    char line[512];
    std::string k;
    cascade_batch_variant tmp{};
    while (fgets(line, sizeof(line), f)) {
      if (!parse_line(line, &k, &tmp)) continue;
      std::string l(line);
      if (!l.empty() && l.back() != '\n') l.push_back('\n');
      if (!lines.count(k)) order.push_back(k);
      lines[k] = l;
    }
    fclose(f);
  }
  char mine[512];
  snprintf(mine, sizeof(mine), "%s\t%d %d %d %d\t%.6g\n", key, v->shape, v->stage, v->prefetch, v->member_cost,
           ns_per_unit);
  if (!lines.count(key)) order.push_back(key);
  lines[key] = mine;
  make_parent_dirs(p);
  char tmpname[1024];
  snprintf(tmpname, sizeof(tmpname), "%s.tmp%ld", p.c_str(), (long)getpid());
  FILE* w = fopen(tmpname, "w");
  if (!w) {
    char msg[256];
    snprintf(msg, sizeof(msg), "tuning cache %s not writable (kept in memory)", p.c_str());
    cpic::set_error_message(msg);
    return CASCADE_OK;
  }
  for (const std::string& k : order) fputs(lines[k].c_str(), w);
  const bool ok = fclose(w) == 0;
  if (!ok || rename(tmpname, p.c_str()) != 0) {
    remove(tmpname);
    cpic::set_error_message("tuning cache: write failed (kept in memory)");
  }
  return CASCADE_OK;
}

const char* cascade_tune_cache_path(void) {
  // per thread, because the name depends on the current device
  thread_local char path[1024];
  path[0] = '\0';
  const char* env = getenv("CASCADE_TUNE_CACHE");
  if (env) {
    snprintf(path, sizeof(path), "%s", env);  // empty: no file, memory only
    return path;
  }
  const char* base = getenv("XDG_CACHE_HOME");
  std::string dir;
  if (base && *base) {
    dir = base;
  } else {
    const char* home = getenv("HOME");
    if (!home || !*home) return path;
    dir = std::string(home) + "/.cache";
  }
  int dev = 0;
  cudaDeviceProp prop{};
  std::string name = "unknown";
  int major = 0, minor = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    name = prop.name;
    major = prop.major;
    minor = prop.minor;
  } else {
    cudaGetLastError();
  }
  for (char& ch : name)
    if (!((ch >= 'a' && ch <= 'z') || (ch >= 'A' && ch <= 'Z') || (ch >= '0' && ch <= '9'))) ch = '_';
  snprintf(path, sizeof(path), "%s/cascade-gb300/batch-tune-%s-sm%d%d.txt", dir.c_str(), name.c_str(), major, minor);
  return path;
}

}  // extern "C"
