// Autotune cache: the tile-shape variant chosen for a (device, lattice,
// storage, layout, size bucket, tile fit) key, kept in a JSON file so that
// later handles skip the timing.
//
// File format (written and read here only):
//   {"version": 1, "entries": {
//    "<key>": {"variant": V, "ms_per_step": M},
//    ...
//   }}
// one entry per line. Unknown lines are kept as they are.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "host.h"

namespace lbm {

namespace {

std::mutex g_mu;
std::string g_path;

bool parse_entry(const std::string& line, std::string& key, int& variant, double& ms)
{
    const size_t k0 = line.find('"');
    if (k0 == std::string::npos) return false;
    const size_t k1 = line.find('"', k0 + 1);
    if (k1 == std::string::npos) return false;
    key = line.substr(k0 + 1, k1 - k0 - 1);
    const size_t v = line.find("\"variant\":", k1);
    const size_t m = line.find("\"ms_per_step\":", k1);
    if (v == std::string::npos || m == std::string::npos) return false;
    variant = std::atoi(line.c_str() + v + 10);
    ms = std::atof(line.c_str() + m + 14);
    return true;
}

std::vector<std::string> read_lines(const std::string& path)
{
    std::vector<std::string> out;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) out.push_back(line);
    return out;
}

}  // namespace

void tune_cache_set_path(const char* path)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_path = path ? path : "";
}

bool tune_cache_lookup(const std::string& key, int* variant, double* ms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_path.empty()) return false;
    for (const std::string& line : read_lines(g_path)) {
        std::string k;
        int v;
        double m;
        if (parse_entry(line, k, v, m) && k == key) {
            *variant = v;
            *ms = m;
            return true;
        }
    }
    return false;
}

void tune_cache_store(const std::string& key, int variant, double ms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_path.empty()) return;
    std::vector<std::string> entries;
    for (const std::string& line : read_lines(g_path)) {
        std::string k;
        int v;
        double m;
        if (parse_entry(line, k, v, m) && k != key) {
            std::string l = line;
            while (!l.empty() && (l.back() == ',' || l.back() == ' ')) l.pop_back();
            entries.push_back(l);
        }
    }
    char buf[512];
    std::snprintf(buf, sizeof(buf), " \"%s\": {\"variant\": %d, \"ms_per_step\": %.6g}", key.c_str(), variant, ms);
    entries.push_back(buf);
    const std::string tmp = g_path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        f << "{\"version\": 1, \"entries\": {\n";
        for (size_t i = 0; i < entries.size(); ++i) f << entries[i] << (i + 1 < entries.size() ? ",\n" : "\n");
        f << "}}\n";
    }
    std::rename(tmp.c_str(), g_path.c_str());
}

}  // namespace lbm
