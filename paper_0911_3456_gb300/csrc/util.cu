// util.cu -- error reporting, environment knobs, device facts and the tuning
// cache of libfbcorr.
//
// Errors follow the paper's requirement that failures surface as recoverable,
// informative conditions rather than aborts (Sec. 5): every entry point returns
// a status and leaves a thread-local message for fbcorr_last_error().
// The tuning cache realises the paper's per-platform, per-input database of
// optimisation configurations (Sec. 6.2): entries are keyed on the GPU name,
// SM count, driver version and the shape/dtype/epilogue key, and stored one
// per line as "key<TAB>value" in <cache dir>/tune.tsv.  Unreadable lines are
// ignored; the file is rewritten atomically.
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "internal.h"

namespace fbc {

namespace {
thread_local char t_err[4096] = "";
std::mutex g_tune_mu;
}  // namespace

fbcorr_status_t set_error(fbcorr_status_t s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof t_err, fmt, ap);
    va_end(ap);
    if (log_enabled()) fprintf(stderr, "[fbcorr] error %d: %s\n", (int)s, t_err);
    return s;
}

void clear_error() { t_err[0] = '\0'; }

const char* last_error_message() { return t_err; }

std::string env_str(const char* name, const char* dflt) {
    const char* v = getenv(name);
    return v ? std::string(v) : std::string(dflt);
}

bool log_enabled() {
    static int on = -1;
    if (on < 0) {
        const std::string v = env_str("FBCORR_LOG", "0");
        on = (!v.empty() && v != "0") ? 1 : 0;
    }
    return on == 1;
}

void logf(const char* fmt, ...) {
    if (!log_enabled()) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[fbcorr] ");
    vfprintf(stderr, fmt, ap);
    fprintf(stderr, "\n");
    va_end(ap);
}

bool fault_injected(const char* what) {
    const std::string v = env_str("FBCORR_FAULT", "");
    return !v.empty() && v.find(what) != std::string::npos;
}

std::string cache_dir() {
    std::string d = env_str("FBCORR_CACHE_DIR", "");
    if (!d.empty()) return d;
    const std::string xdg = env_str("XDG_CACHE_HOME", "");
    if (!xdg.empty()) return xdg + "/fbcorr";
    const std::string home = env_str("HOME", "/tmp");
    return home + "/.cache/fbcorr";
}

fbcorr_status_t device_info(DeviceInfo* out) {
    DeviceInfo d;
    FBC_CUDA(cudaGetDevice(&d.device));
    cudaDeviceProp prop;
    FBC_CUDA(cudaGetDeviceProperties(&prop, d.device));
    d.sm_count = prop.multiProcessorCount;
    d.cc_major = prop.major;
    d.cc_minor = prop.minor;
    d.smem_optin = prop.sharedMemPerBlockOptin;
    snprintf(d.name, sizeof d.name, "%s", prop.name);
    FBC_CUDA(cudaDriverGetVersion(&d.driver_version));
    *out = d;
    return FBCORR_OK;
}

std::string tune_key(const DeviceInfo& dev, const std::string& what) {
    std::ostringstream o;
    std::string name = dev.name;
    for (auto& ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    o << name << "|sm" << dev.sm_count << "|cc" << dev.cc_major << dev.cc_minor << "|drv"
      << dev.driver_version << "|" << what;
    return o.str();
}

namespace {
std::string tune_path() { return cache_dir() + "/tune.tsv"; }

std::map<std::string, std::string> tune_read() {
    std::map<std::string, std::string> m;
    std::ifstream f(tune_path());
    std::string line;
    while (std::getline(f, line)) {
        const size_t t = line.find('\t');
        if (t == std::string::npos || t == 0 || t + 1 >= line.size()) continue;   // corrupt line
        m[line.substr(0, t)] = line.substr(t + 1);
    }
    return m;
}
}  // namespace

bool tune_lookup(const std::string& key, std::string* value) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto m = tune_read();
    auto it = m.find(key);
    if (it == m.end()) return false;
    *value = it->second;
    return true;
}

void tune_store(const std::string& key, const std::string& value) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto m = tune_read();
    m[key] = value;
    const std::string dir = cache_dir();
    std::string cur;
    for (size_t i = 0; i < dir.size(); ++i) {
        cur += dir[i];
        if (dir[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
    }
    mkdir(dir.c_str(), 0755);
    const std::string path = tune_path();
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    {
        std::ofstream f(tmp, std::ios::trunc);
        for (auto& kv : m) f << kv.first << '\t' << kv.second << '\n';
        if (!f.good()) {
            unlink(tmp.c_str());
            return;
        }
    }
    rename(tmp.c_str(), path.c_str());
}

}  // namespace fbc
