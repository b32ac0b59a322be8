// rtcg.cu -- run-time code generation: NVRTC compile for sm_103a, an on-disk
// cubin cache, and module loading through the CUDA driver API.
//
// The paper builds its kernels from source strings at run time and caches the
// binaries in a "semi-permanent" compiler cache keyed on the hardware/software
// environment, recompiling only when that changes (Sec. 5, Fig. 2).  Here the
// cache key is a hash of the full source, the NVRTC options, the NVRTC
// version and the target architecture; the file is written atomically
// (temporary file + rename) so that concurrent processes never read a torn
// binary.  Driver entry points are resolved through the runtime, so the
// library does not link libcuda and still loads on machines without a GPU.
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

#include "internal.h"

namespace fbc {

namespace {

struct DriverApi {
    bool ok = false;
    CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
    CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
    CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned,
                             unsigned, unsigned, CUstream, void**, void**) = nullptr;
    CUresult (*ctxGetCurrent)(CUcontext*) = nullptr;
    CUresult (*getErrorString)(CUresult, const char**) = nullptr;
    CUresult (*graphAddKernelNode)(CUgraphNode*, CUgraph, const CUgraphNode*, size_t,
                                   const CUDA_KERNEL_NODE_PARAMS*) = nullptr;
    CUresult (*graphExecKernelNodeSetParams)(CUgraphExec, CUgraphNode,
                                             const CUDA_KERNEL_NODE_PARAMS*) = nullptr;
    CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
    CUresult (*launchKernelEx)(const CUlaunchConfig*, CUfunction, void**, void**) = nullptr;   // optional
    CUresult (*funcGetAttribute)(int*, CUfunction_attribute, CUfunction) = nullptr;            // optional
};

std::mutex g_mu;
DriverApi g_drv;

template <typename F>
bool resolve(const char* sym, F* fp) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(sym, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *fp = reinterpret_cast<F>(p);
    return true;
}

fbcorr_status_t driver_api(DriverApi** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_drv.ok) {
        DriverApi d;
        bool ok = resolve("cuModuleLoadData", &d.moduleLoadData) &&
                  resolve("cuModuleGetFunction", &d.moduleGetFunction) &&
                  resolve("cuFuncSetAttribute", &d.funcSetAttribute) &&
                  resolve("cuLaunchKernel", &d.launchKernel) &&
                  resolve("cuCtxGetCurrent", &d.ctxGetCurrent) &&
                  resolve("cuGetErrorString", &d.getErrorString) &&
                  resolve("cuGraphAddKernelNode", &d.graphAddKernelNode) &&
                  resolve("cuGraphExecKernelNodeSetParams", &d.graphExecKernelNodeSetParams) &&
                  resolve("cuOccupancyMaxActiveBlocksPerMultiprocessor", &d.occupancy);
        if (!ok) return set_error(FBCORR_ERR_CUDA, "could not resolve CUDA driver entry points");
        if (!resolve("cuLaunchKernelEx", &d.launchKernelEx)) d.launchKernelEx = nullptr;
        if (!resolve("cuFuncGetAttribute", &d.funcGetAttribute)) d.funcGetAttribute = nullptr;
        d.ok = true;
        g_drv = d;
    }
    *out = &g_drv;
    return FBCORR_OK;
}

const char* cu_err(CUresult r) {
    const char* s = "unknown driver error";
    if (g_drv.getErrorString) g_drv.getErrorString(r, &s);
    return s;
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

const char* kArch = "sm_103a";

std::vector<std::string> nvrtc_options() {
    return {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DFBC_NVRTC=1"};
}

std::string nvrtc_version_string() {
    int maj = 0, min = 0;
    nvrtcVersion(&maj, &min);
    char b[32];
    snprintf(b, sizeof b, "%d.%d", maj, min);
    return b;
}

fbcorr_status_t compile(const std::string& src, std::vector<char>* cubin, std::string* log) {
    if (fault_injected("nvrtc"))
        return set_error(FBCORR_ERR_NVRTC, "NVRTC compilation disabled by FBCORR_FAULT=nvrtc");
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "fbcorr_rtcg.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS)
        return set_error(FBCORR_ERR_NVRTC, "nvrtcCreateProgram: %s", nvrtcGetErrorString(r));
    std::vector<std::string> opts = nvrtc_options();
    std::vector<const char*> copts;
    for (auto& o : opts) copts.push_back(o.c_str());
    r = nvrtcCompileProgram(prog, (int)copts.size(), copts.data());
    size_t logsz = 0;
    nvrtcGetProgramLogSize(prog, &logsz);
    std::string lg(logsz, '\0');
    if (logsz) nvrtcGetProgramLog(prog, &lg[0]);
    if (log) *log = lg;
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return set_error(FBCORR_ERR_NVRTC, "NVRTC compile failed: %s\n%.2000s",
                         nvrtcGetErrorString(r), lg.c_str());
    }
    size_t n = 0;
    if (nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
        nvrtcDestroyProgram(&prog);
        return set_error(FBCORR_ERR_NVRTC, "NVRTC produced no cubin");
    }
    cubin->resize(n);
    nvrtcGetCUBIN(prog, cubin->data());
    nvrtcDestroyProgram(&prog);
    return FBCORR_OK;
}

bool read_file(const std::string& path, std::vector<char>* out) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return false;
    fseek(f, 0, SEEK_END);
    long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    if (n <= 0) {
        fclose(f);
        return false;
    }
    out->resize((size_t)n);
    bool ok = fread(out->data(), 1, (size_t)n, f) == (size_t)n;
    fclose(f);
    return ok;
}

void mkdirs(const std::string& dir) {
    std::string cur;
    for (size_t i = 0; i < dir.size(); ++i) {
        cur += dir[i];
        if (dir[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
    }
    mkdir(dir.c_str(), 0755);
}

void write_file_atomic(const std::string& path, const std::vector<char>& data) {
    std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
    ok = (fclose(f) == 0) && ok;
    if (ok)
        rename(tmp.c_str(), path.c_str());
    else
        unlink(tmp.c_str());
}

struct ModKey {
    CUcontext ctx;
    uint64_t hash;
    bool operator<(const ModKey& o) const {
        return ctx != o.ctx ? ctx < o.ctx : hash < o.hash;
    }
};
std::map<ModKey, CUmodule> g_modules;   // loaded once per context, kept for the process

}  // namespace

// FBCORR_DUMP_DIR: write every generated source there (for offline ptxas -v checks).
void dump_source(const std::string& src, const std::string& name) {
    const std::string dir = env_str("FBCORR_DUMP_DIR", "");
    if (dir.empty()) return;
    mkdirs(dir);
    FILE* f = fopen((dir + "/" + name + ".cu").c_str(), "w");
    if (!f) return;
    fwrite(src.data(), 1, src.size(), f);
    fclose(f);
}

fbcorr_status_t rtcg_compile_only(const std::string& src, std::string* log) {
    std::vector<char> cubin;
    dump_source(src, "check_" + std::to_string(fnv1a(src) & 0xffffff));
    return compile(src, &cubin, log);
}

namespace {
uint64_t source_hash(const std::string& src) {
    std::string keysrc = src + "\n//" + kArch + " nvrtc " + nvrtc_version_string();
    for (auto& o : nvrtc_options()) keysrc += " " + o;
    return fnv1a(keysrc);
}

std::string cubin_path(uint64_t h) {
    char hb[32];
    snprintf(hb, sizeof hb, "%016llx", (unsigned long long)h);
    return cache_dir() + "/rtcg-" + hb + ".cubin";
}
}  // namespace

fbcorr_status_t rtcg_precompile(const std::vector<std::string>& sources) {
    // Compile on host threads every source whose cubin is not cached yet; the
    // results land in the on-disk cache that rtcg_kernel reads.  Failures are
    // left for rtcg_kernel to report.
    if (fault_injected("nvrtc") || fault_injected("nocache")) return FBCORR_OK;
    std::vector<const std::string*> todo;
    for (const auto& src : sources) {
        struct stat st;
        if (stat(cubin_path(source_hash(src)).c_str(), &st) != 0) todo.push_back(&src);
    }
    if (todo.empty()) return FBCORR_OK;
    mkdirs(cache_dir());
    unsigned hw = std::thread::hardware_concurrency();
    const size_t nthreads = std::min<size_t>(todo.size(), std::max(1u, std::min(hw ? hw : 4u, 32u)));
    std::atomic<size_t> next{0};
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthreads; ++t)
        pool.emplace_back([&]() {
            for (size_t k = next++; k < todo.size(); k = next++) {
                std::vector<char> cubin;
                std::string lg;
                if (compile(*todo[k], &cubin, &lg) == FBCORR_OK)
                    write_file_atomic(cubin_path(source_hash(*todo[k])), cubin);
            }
        });
    for (auto& th : pool) th.join();
    logf("rtcg: precompiled %zu sources on %zu threads", todo.size(), nthreads);
    clear_error();
    return FBCORR_OK;
}

fbcorr_status_t rtcg_kernel(const std::string& src, const std::string& name, size_t smem,
                            int threads, Kernel* out) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    FBC_CUDA(cudaFree(nullptr));   // make the primary context current
    CUcontext ctx = nullptr;
    if (drv->ctxGetCurrent(&ctx) != CUDA_SUCCESS || !ctx)
        return set_error(FBCORR_ERR_CUDA, "no current CUDA context");

    const uint64_t h = source_hash(src);

    CUmodule mod = nullptr;
    const bool nocache = fault_injected("nocache");   // testing knob: bypass both caches
    if (!nocache) {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_modules.find(ModKey{ctx, h});
        if (it != g_modules.end()) mod = it->second;
    }
    if (!mod) {
        const std::string dir = cache_dir();
        const std::string path = cubin_path(h);
        std::vector<char> cubin;
        bool cached = !nocache && read_file(path, &cubin);
        if (!cached) {
            dump_source(src, name);
            FBC_TRY(compile(src, &cubin, nullptr));
            mkdirs(dir);
            write_file_atomic(path, cubin);
            logf("rtcg: compiled %s (%zu bytes) -> %s", name.c_str(), cubin.size(), path.c_str());
        } else {
            logf("rtcg: cache hit %s for %s", path.c_str(), name.c_str());
        }
        CUresult r = drv->moduleLoadData(&mod, cubin.data());
        if (r != CUDA_SUCCESS && cached) {
            // stale or corrupt cache entry: rebuild it once
            FBC_TRY(compile(src, &cubin, nullptr));
            write_file_atomic(path, cubin);
            r = drv->moduleLoadData(&mod, cubin.data());
        }
        if (r != CUDA_SUCCESS)
            return set_error(FBCORR_ERR_CUDA, "cuModuleLoadData(%s): %s", name.c_str(), cu_err(r));
        std::lock_guard<std::mutex> lk(g_mu);
        g_modules[ModKey{ctx, h}] = mod;
    }
    CUfunction fn = nullptr;
    CUresult r = drv->moduleGetFunction(&fn, mod, name.c_str());
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuModuleGetFunction(%s): %s", name.c_str(), cu_err(r));
    if (smem > 48 * 1024) {
        r = drv->funcSetAttribute(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem);
        if (r != CUDA_SUCCESS)
            return set_error(FBCORR_ERR_CUDA, "cuFuncSetAttribute(smem=%zu): %s", smem, cu_err(r));
    }
    out->fn = fn;
    out->threads = threads;
    out->smem = smem;
    out->name = name;
    out->src_hash = h;
    return FBCORR_OK;
}

std::string hex64(unsigned long long v) {
    char b[32];
    snprintf(b, sizeof b, "%016llx", v);
    return b;
}

bool encode_f32_store_map(void* map, const float* base, const unsigned long long dims[3],
                          const unsigned long long strides[2], const unsigned box[3]) {
    // resolved on first use and kept out of driver_api(): a driver without tensor
    // maps leaves the caller on its direct-store path
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn fn = nullptr;
    static bool tried = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!tried) {
            tried = true;
            if (!resolve("cuTensorMapEncodeTiled", &fn)) fn = nullptr;
        }
    }
    if (!fn) return false;
    const cuuint64_t gdim[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t gstride[2] = {strides[0], strides[1]};
    const cuuint32_t bdim[3] = {box[0], box[1], box[2]};
    const cuuint32_t estride[3] = {1, 1, 1};
    return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), gdim,
              gstride, bdim, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

fbcorr_status_t launch(const Kernel& k, dim3 grid, void** args, cudaStream_t stream) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    if (!k.fn) return set_error(FBCORR_ERR_INTERNAL, "launch of an unloaded kernel");
    CUresult r = drv->launchKernel(k.fn, grid.x, grid.y, grid.z, (unsigned)k.threads, 1, 1,
                                   (unsigned)k.smem, (CUstream)stream, args, nullptr);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuLaunchKernel(%s grid=%u,%u,%u block=%d smem=%zu): %s",
                         k.name.c_str(), grid.x, grid.y, grid.z, k.threads, k.smem, cu_err(r));
    return FBCORR_OK;
}

fbcorr_status_t launch_dependent(const Kernel& k, dim3 grid, void** args, cudaStream_t stream) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    if (!drv->launchKernelEx) return launch(k, grid, args, stream);
    if (!k.fn) return set_error(FBCORR_ERR_INTERNAL, "launch of an unloaded kernel");
    CUlaunchAttribute attr;
    memset(&attr, 0, sizeof attr);
    attr.id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
    attr.value.programmaticStreamSerializationAllowed = 1;
    CUlaunchConfig cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDimX = grid.x;
    cfg.gridDimY = grid.y;
    cfg.gridDimZ = grid.z;
    cfg.blockDimX = (unsigned)k.threads;
    cfg.blockDimY = 1;
    cfg.blockDimZ = 1;
    cfg.sharedMemBytes = (unsigned)k.smem;
    cfg.hStream = (CUstream)stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    CUresult r = drv->launchKernelEx(&cfg, k.fn, args, nullptr);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuLaunchKernelEx(%s grid=%u block=%d smem=%zu, dependent): %s",
                         k.name.c_str(), grid.x, k.threads, k.smem, cu_err(r));
    return FBCORR_OK;
}

namespace {
CUDA_KERNEL_NODE_PARAMS node_params(const Kernel& k, dim3 grid, void** args) {
    CUDA_KERNEL_NODE_PARAMS np;
    memset(&np, 0, sizeof np);
    np.func = k.fn;
    np.gridDimX = grid.x;
    np.gridDimY = grid.y;
    np.gridDimZ = grid.z;
    np.blockDimX = (unsigned)k.threads;
    np.blockDimY = 1;
    np.blockDimZ = 1;
    np.sharedMemBytes = (unsigned)k.smem;
    np.kernelParams = args;
    np.extra = nullptr;
    return np;
}
}  // namespace

fbcorr_status_t graph_add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                                 const Kernel& k, dim3 grid, void** args, cudaGraphNode_t* out) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    const CUDA_KERNEL_NODE_PARAMS np = node_params(k, grid, args);
    CUresult r = drv->graphAddKernelNode((CUgraphNode*)out, (CUgraph)g, (const CUgraphNode*)deps,
                                         ndeps, &np);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuGraphAddKernelNode(%s): %s", k.name.c_str(), cu_err(r));
    return FBCORR_OK;
}

fbcorr_status_t graph_set_kernel(cudaGraphExec_t e, cudaGraphNode_t n, const Kernel& k, dim3 grid,
                                 void** args) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    const CUDA_KERNEL_NODE_PARAMS np = node_params(k, grid, args);
    CUresult r = drv->graphExecKernelNodeSetParams((CUgraphExec)e, (CUgraphNode)n, &np);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuGraphExecKernelNodeSetParams(%s): %s", k.name.c_str(),
                         cu_err(r));
    return FBCORR_OK;
}

fbcorr_status_t kernel_resources(const Kernel& k, int* regs, int* local_bytes) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    if (!drv->funcGetAttribute) return set_error(FBCORR_ERR_CUDA, "cuFuncGetAttribute unavailable");
    CUresult r = drv->funcGetAttribute(regs, CU_FUNC_ATTRIBUTE_NUM_REGS, k.fn);
    if (r == CUDA_SUCCESS) r = drv->funcGetAttribute(local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, k.fn);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuFuncGetAttribute(%s): %s", k.name.c_str(), cu_err(r));
    return FBCORR_OK;
}

fbcorr_status_t kernel_occupancy(const Kernel& k, int* blocks_per_sm) {
    DriverApi* drv = nullptr;
    FBC_TRY(driver_api(&drv));
    CUresult r = drv->occupancy(blocks_per_sm, k.fn, k.threads, k.smem);
    if (r != CUDA_SUCCESS)
        return set_error(FBCORR_ERR_CUDA, "cuOccupancyMaxActiveBlocksPerMultiprocessor(%s): %s",
                         k.name.c_str(), cu_err(r));
    return FBCORR_OK;
}

}  // namespace fbc
