// Launch-shape tuner cache: key -> (a, b, c).  Entries live in memory and, when
// possible, in a text file (one "key a b c" line per entry) so that a shape
// measured once is reused by later processes.  The file is
// $SNSOLVE_TUNE_CACHE, else $HOME/.cache/snsolve_tune.txt; if neither can be
// written the cache is kept in memory only.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <sys/types.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

namespace sns {

static std::mutex g_mu;
static std::map<std::string, std::tuple<int, int, int>> g_cache;
static bool g_loaded = false;

static std::string cache_path() {
  const char* e = getenv("SNSOLVE_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  if (h && *h) return std::string(h) + "/.cache/snsolve_tune.txt";
  return "";
}

static void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string p = cache_path();
  if (p.empty()) return;
  FILE* f = fopen(p.c_str(), "r");
  if (!f) return;
  char key[256];
  int a, b, c;
  while (fscanf(f, "%255s %d %d %d", key, &a, &b, &c) == 4) g_cache[key] = std::make_tuple(a, b, c);
  fclose(f);
}

bool tune_lookup(const char* key, int* a, int* b, int* c) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  std::tie(*a, *b, *c) = it->second;
  return true;
}

void tune_store(const char* key, int a, int b, int c) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  g_cache[key] = std::make_tuple(a, b, c);
  const std::string p = cache_path();
  if (p.empty()) return;
  const size_t slash = p.find_last_of('/');
  if (slash != std::string::npos && slash > 0) mkdir(p.substr(0, slash).c_str(), 0755);   // best effort
  FILE* f = fopen(p.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", key, a, b, c);
  fclose(f);
}

}  // namespace sns

extern "C" {
// Clears the in-memory tuner cache (the file is left alone).
void snsolve_tune_reset(void) {
  std::lock_guard<std::mutex> lk(sns::g_mu);
  sns::g_cache.clear();
  sns::g_loaded = true;
}
}
