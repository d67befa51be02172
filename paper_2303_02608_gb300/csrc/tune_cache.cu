// Autotuning cache: one "key value" line per tuned choice in a small text file
// ($ESIM_AD_CACHE, default ~/.cache/esim_ad_autotune.txt).  The last line for a
// key wins.  The cache is an optimisation only: any I/O failure is ignored.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace esim {
namespace {

std::mutex g_cache_mu;

std::string cache_path()
{
    if (const char* p = getenv("ESIM_AD_CACHE")) return p;
    const char* home = getenv("HOME");
    return std::string(home ? home : ".") + "/.cache/esim_ad_autotune.txt";
}

}  // namespace

int tune_cache_lookup(const char* key)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE* f = fopen(cache_path().c_str(), "r");
    if (!f) return 0;
    const size_t L = strlen(key);
    char line[256];
    int found = 0;
    while (fgets(line, sizeof(line), f))
        if (strncmp(line, key, L) == 0 && line[L] == ' ') found = atoi(line + L + 1);
    fclose(f);
    return found;
}

void tune_cache_store(const char* key, int value)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const std::string path = cache_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);   // may already exist
    FILE* f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key, value);
    fclose(f);
}

}  // namespace esim
