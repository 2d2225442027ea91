// user.cu -- user-supplied functions: the user's f, written once as a
// template on the number type, is compiled at run time with NVRTC for sm_103a
// together with the library's hDual operators (user_num.cuh) and the CHESS-VEC
// / CHUNK-HESS sweep (user_kernel.cuh), loaded as a CUDA library, and launched
// on the caller's stream.  The paper's premise (Sec. I, Sec. IV) is that the
// user overloads f on hDual; a compiled C ABI cannot instantiate a template at
// the caller's site, so the instantiation happens here, once per handle.
//
// NVRTC is opened with dlopen on first use, so the rest of the library does not
// depend on it; without it chessfad_user_fn_create returns CHESSFAD_ERR_JIT.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/chessfad.h"
#include "user_embed.h"  // generated by the build: kHdualSrc, kSymLayoutSrc, kUserNumSrc, kUserKernelSrc

struct chessfad_user_fn {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t hvp = nullptr;          // plain (CHESS-VEC, Alg. 7)
    cudaKernel_t hessian = nullptr;      // plain (CHUNK-HESS, Alg. 5)
    cudaKernel_t sym_hvp = nullptr;      // symmetric (SC-HESS-VEC, Alg. 8)
    cudaKernel_t sym_hessian = nullptr;  // symmetric (SCHUNK-HESS, Alg. 6)
    cudaKernel_t hvp_n1 = nullptr;       // FP32 handles, n = 1: FP64 arithmetic, float I/O
    cudaKernel_t hessian_n1 = nullptr;
    int csize = 0;
    int prec = 0;
    std::mutex mu;
    unsigned long long smem_opted = 0;  // bit d: the symmetric kernels' shared-memory limit raised on device d
};

namespace {

struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    const char *(*error_string)(nvrtcResult) = nullptr;
};

std::mutex g_nvrtc_mu;
Nvrtc g_nvrtc;
bool g_nvrtc_tried = false;

const Nvrtc &nvrtc()
{
    std::lock_guard<std::mutex> lk(g_nvrtc_mu);
    if (g_nvrtc_tried) return g_nvrtc;
    g_nvrtc_tried = true;
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char *env : {"CUDA_HOME", "CUDA_PATH"}) {
        const char *root = std::getenv(env);
        if (root && *root) names.push_back(std::string(root) + "/lib64/libnvrtc.so.13");
    }
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void *h = nullptr;
    for (const auto &nm : names)
        if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
        g_nvrtc.why = "NVRTC (libnvrtc.so.13) not found";
        return g_nvrtc;
    }
    auto sym = [&](const char *s) { return dlsym(h, s); };
    g_nvrtc.create = reinterpret_cast<decltype(g_nvrtc.create)>(sym("nvrtcCreateProgram"));
    g_nvrtc.compile = reinterpret_cast<decltype(g_nvrtc.compile)>(sym("nvrtcCompileProgram"));
    g_nvrtc.log_size = reinterpret_cast<decltype(g_nvrtc.log_size)>(sym("nvrtcGetProgramLogSize"));
    g_nvrtc.log = reinterpret_cast<decltype(g_nvrtc.log)>(sym("nvrtcGetProgramLog"));
    g_nvrtc.cubin_size = reinterpret_cast<decltype(g_nvrtc.cubin_size)>(sym("nvrtcGetCUBINSize"));
    g_nvrtc.cubin = reinterpret_cast<decltype(g_nvrtc.cubin)>(sym("nvrtcGetCUBIN"));
    g_nvrtc.destroy = reinterpret_cast<decltype(g_nvrtc.destroy)>(sym("nvrtcDestroyProgram"));
    g_nvrtc.error_string = reinterpret_cast<decltype(g_nvrtc.error_string)>(sym("nvrtcGetErrorString"));
    g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.log_size && g_nvrtc.log && g_nvrtc.cubin_size &&
                 g_nvrtc.cubin && g_nvrtc.destroy && g_nvrtc.error_string;
    if (!g_nvrtc.ok) g_nvrtc.why = "NVRTC library lacks an expected entry point";
    return g_nvrtc;
}

void put_log(char *log, size_t log_bytes, const std::string &text)
{
    if (!log || log_bytes == 0) return;
    const size_t k = text.size() < log_bytes - 1 ? text.size() : log_bytes - 1;
    std::memcpy(log, text.data(), k);
    log[k] = '\0';
}

bool is_identifier(const char *s)
{
    if (!s || !(std::isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
    for (const char *p = s; *p; ++p)
        if (!(std::isalnum((unsigned char)*p) || *p == '_')) return false;
    return true;
}

bool valid_chunk(int c) { return c == 1 || c == 2 || c == 4 || c == 8 || c == 16 || c == 32; }

constexpr int kBlock = 256;
constexpr size_t kSmemBudget = 200 * 1024;  // symmetric kernels' dynamic shared memory ceiling

struct UserArgs {  // the kernels' chessfad::user::UserArgs, field for field
    const void *x;
    const void *v;
    void *out;
    long long batch;
    const double *params;
    int n;
    int maxpts;
    int tpp;
    int acc;
};

long long hs_elems(int n, int C)  // staged chunk matrix of one point, symmetric HVP
{
    const long long nch = (n + C - 1) / C;
    return C * (nch * (n + 1) - C * nch * (nch - 1) / 2);
}

// Resolve a launch configuration for a handle: method 0 = plain, 1 =
// symmetric; -1 = symmetric when its shared memory fits, else plain.
int resolve(const chessfad_user_fn *fn, const chessfad_config *cfg, bool hvp, int n, long long batch, int &method,
            int &bt, int &tpp, int &ppb, size_t &smem, int &acc)
{
    const size_t elem = fn->prec == CHESSFAD_FP64 ? sizeof(double) : sizeof(float);
    method = -1;
    bt = 0;
    tpp = 0;
    acc = 0;
    if (cfg) {
        if (cfg->csize != 0 && cfg->csize != fn->csize) return CHESSFAD_ERR_CHUNK;
        if (cfg->method != CHESSFAD_METHOD_PLAIN && cfg->method != CHESSFAD_METHOD_SYMMETRIC) return CHESSFAD_ERR_CONFIG;
        if (cfg->threads_per_row > 1) return CHESSFAD_ERR_CONFIG;
        if (cfg->block_threads != 0 && (cfg->block_threads < 32 || cfg->block_threads > 256 || cfg->block_threads % 32))
            return CHESSFAD_ERR_CONFIG;
        const int p = cfg->threads_per_point;
        if (p != 0 && (p < 32 || p > 256 || (p & (p - 1)))) return CHESSFAD_ERR_CONFIG;
        method = cfg->method;
        bt = cfg->block_threads;
        tpp = p;
    }
    if (bt == 0) bt = kBlock;
    if (tpp == 0) tpp = 32;
    if (method != CHESSFAD_METHOD_PLAIN) {
        if (tpp > bt) bt = tpp;
        // staged chunk matrix, else (HVP) FP64 row accumulators
        for (int form = 0; form < (hvp ? 2 : 1); ++form) {
            // form 1 (accumulators): per point n FP64 accumulators, x, v and
            // the per-iteration stage of its threads (C values, an FP64 row
            // dot and two ints each), plus 32 bytes of alignment
            const size_t per_pt = form == 0 ? ((size_t)n * (hvp ? 2 : 1) + (hvp ? (size_t)hs_elems(n, fn->csize) : 0)) * elem
                                            : (size_t)n * 2 * elem + (size_t)n * sizeof(double) +
                                                  (size_t)tpp * ((size_t)fn->csize * elem + sizeof(double) + 2 * sizeof(int)) + 32;
            long long p = bt / tpp;
            if (p > batch) p = batch;
            while (p > 1 && (size_t)p * per_pt > kSmemBudget) --p;
            if ((size_t)p * per_pt <= kSmemBudget) {
                method = CHESSFAD_METHOD_SYMMETRIC;
                ppb = (int)p;
                smem = (size_t)p * per_pt;
                acc = form;
                return CHESSFAD_SUCCESS;
            }
        }
        if (method == CHESSFAD_METHOD_SYMMETRIC) return CHESSFAD_ERR_SIZE;
    }
    method = CHESSFAD_METHOD_PLAIN;
    const long long per_cta = (bt - 1) / n + 2;
    ppb = (int)(batch < per_cta ? batch : per_cta);
    smem = (size_t)ppb * n * elem * 2;
    return CHESSFAD_SUCCESS;
}

int launch(chessfad_user_fn *fn, const chessfad_config *cfg, bool hvp, int n, long long batch, const void *x,
           const void *v, void *out, const double *params, cudaStream_t stream)
{
    if (!fn || !fn->lib) return CHESSFAD_ERR_NULL;
    if (n < 1 || n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
    if (batch < 0) return CHESSFAD_ERR_BATCH;
    int method, bt, tpp, ppb = 0, acc = 0;
    size_t smem = 0;
    int st = resolve(fn, cfg, hvp, n, batch > 0 ? batch : 1, method, bt, tpp, ppb, smem, acc);
    if (st != CHESSFAD_SUCCESS) return st;
    if (batch == 0) return CHESSFAD_SUCCESS;
    if (!x || !out || (hvp && !v)) return CHESSFAD_ERR_NULL;
    UserArgs args{x, hvp ? v : x, out, batch, params, n, ppb, tpp, acc};
    long long grid;
    unsigned block;
    cudaKernel_t k;
    if (fn->prec == CHESSFAD_FP32_COMP && n == 1) {
        // one variable: the FP64 kernel with float I/O (a single Hessian
        // entry whose terms can cancel), by the plain decomposition (the
        // symmetric one has the same single item)
        const int b = bt > 0 ? bt : kBlock;
        const long long per_cta = b + 1;
        args.maxpts = (int)(batch < per_cta ? batch : per_cta);
        args.tpp = 1;
        args.acc = 0;
        grid = (batch + b - 1) / b;
        block = (unsigned)b;
        smem = (size_t)args.maxpts * 2 * sizeof(double);
        k = hvp ? fn->hvp_n1 : fn->hessian_n1;
    } else if (method == CHESSFAD_METHOD_SYMMETRIC) {
        grid = (batch + ppb - 1) / ppb;
        block = (unsigned)(ppb * tpp);
        k = hvp ? fn->sym_hvp : fn->sym_hessian;
        if (smem > 48 * 1024) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
            std::lock_guard<std::mutex> lk(fn->mu);
            const unsigned long long bit = 1ull << (dev & 63);
            if (!(fn->smem_opted & bit)) {
                for (cudaKernel_t kk : {fn->sym_hvp, fn->sym_hessian})
                    if (cudaFuncSetAttribute(reinterpret_cast<const void *>(kk),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) !=
                        cudaSuccess)
                        return CHESSFAD_ERR_CUDA;
                fn->smem_opted |= bit;
            }
        }
    } else {
        grid = (batch * (long long)n + bt - 1) / bt;
        block = (unsigned)bt;
        k = hvp ? fn->hvp : fn->hessian;
    }
    if (grid > 0x7fffffffLL) return CHESSFAD_ERR_BATCH;
    void *argv[] = {&args};
    cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void *>(k), dim3((unsigned)grid), dim3(block), argv, smem,
                                     stream);
    return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

}  // namespace

extern "C" {

CHESSFAD_API int chessfad_user_fn_create(const char *source, const char *name, int csize, int prec,
                                         chessfad_user_fn **out, char *log, size_t log_bytes)
{
    put_log(log, log_bytes, "");
    if (!source || !name || !out) return CHESSFAD_ERR_NULL;
    *out = nullptr;
    if (!valid_chunk(csize)) return CHESSFAD_ERR_CHUNK;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (!is_identifier(name)) {
        put_log(log, log_bytes, "function name is not a C identifier");
        return CHESSFAD_ERR_JIT;
    }
    const Nvrtc &rt = nvrtc();
    if (!rt.ok) {
        put_log(log, log_bytes, rt.why);
        return CHESSFAD_ERR_JIT;
    }
    std::string text = "#include \"user_num.cuh\"\n#line 1 \"user_function\"\n";
    text += source;
    text += "\n#include \"user_kernel.cuh\"\n";
    const char *headers[] = {kHdualSrc, kSymLayoutSrc, kUserNumSrc, kUserKernelSrc, ""};
    const char *header_names[] = {"hdual.cuh", "sym_layout.cuh", "user_num.cuh", "user_kernel.cuh", "cuda_runtime.h"};
    nvrtcProgram prog = nullptr;
    if (rt.create(&prog, text.c_str(), "chessfad_user.cu", 5, headers, header_names) != NVRTC_SUCCESS) {
        put_log(log, log_bytes, "nvrtcCreateProgram failed");
        return CHESSFAD_ERR_JIT;
    }
    const std::string def_t = std::string("-DCHESSFAD_USER_T=") + (prec == CHESSFAD_FP64 ? "double" : "float");
    const std::string def_c = "-DCHESSFAD_USER_C=" + std::to_string(csize);
    const std::string def_fn = std::string("-DCHESSFAD_USER_FN=") + name;
    const std::string def_f32 = std::string("-DCHESSFAD_USER_F32=") + (prec == CHESSFAD_FP64 ? "0" : "1");
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device",
                          def_t.c_str(), def_c.c_str(), def_fn.c_str(), def_f32.c_str()};
    const nvrtcResult cr = rt.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    size_t lsz = 0;
    rt.log_size(prog, &lsz);
    std::string ltext(lsz, '\0');
    if (lsz > 0) rt.log(prog, &ltext[0]);
    while (!ltext.empty() && ltext.back() == '\0') ltext.pop_back();
    if (cr != NVRTC_SUCCESS) {
        put_log(log, log_bytes, std::string(rt.error_string(cr)) + "\n" + ltext);
        rt.destroy(&prog);
        return CHESSFAD_ERR_JIT;
    }
    put_log(log, log_bytes, ltext);
    size_t csz = 0;
    rt.cubin_size(prog, &csz);
    std::vector<char> cubin(csz);
    if (csz == 0 || rt.cubin(prog, cubin.data()) != NVRTC_SUCCESS) {
        rt.destroy(&prog);
        put_log(log, log_bytes, "NVRTC produced no cubin");
        return CHESSFAD_ERR_JIT;
    }
    rt.destroy(&prog);

    auto *fn = new chessfad_user_fn;
    fn->csize = csize;
    fn->prec = prec;
    cudaError_t e = cudaLibraryLoadData(&fn->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&fn->hvp, fn->lib, "chessfad_user_hvp");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&fn->hessian, fn->lib, "chessfad_user_hessian");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&fn->sym_hvp, fn->lib, "chessfad_user_sym_hvp");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&fn->sym_hessian, fn->lib, "chessfad_user_sym_hessian");
    if (e == cudaSuccess && prec == CHESSFAD_FP32_COMP) e = cudaLibraryGetKernel(&fn->hvp_n1, fn->lib, "chessfad_user_hvp_n1");
    if (e == cudaSuccess && prec == CHESSFAD_FP32_COMP)
        e = cudaLibraryGetKernel(&fn->hessian_n1, fn->lib, "chessfad_user_hessian_n1");
    if (e != cudaSuccess) {
        cudaGetLastError();
        put_log(log, log_bytes, std::string("compiled; loading failed: ") + cudaGetErrorString(e));
        if (fn->lib) cudaLibraryUnload(fn->lib);
        delete fn;
        return CHESSFAD_ERR_CUDA;
    }
    *out = fn;
    return CHESSFAD_SUCCESS;
}

CHESSFAD_API int chessfad_user_fn_destroy(chessfad_user_fn *fn)
{
    if (!fn) return CHESSFAD_SUCCESS;
    cudaError_t e = fn->lib ? cudaLibraryUnload(fn->lib) : cudaSuccess;
    delete fn;
    return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

CHESSFAD_API int chessfad_user_fn_info(const chessfad_user_fn *fn, int hvp, int *csize, int *prec, int *registers,
                                       int *local_bytes)
{
    if (!fn || !fn->lib) return CHESSFAD_ERR_NULL;
    if (csize) *csize = fn->csize;
    if (prec) *prec = fn->prec;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(hvp ? fn->hvp : fn->hessian)) != cudaSuccess)
        return CHESSFAD_ERR_CUDA;
    if (registers) *registers = fa.numRegs;
    if (local_bytes) *local_bytes = (int)fa.localSizeBytes;
    return CHESSFAD_SUCCESS;
}

CHESSFAD_API int chessfad_user_hvp(chessfad_user_fn *fn, int n, long long batch, const void *x, const void *v,
                                   void *out, const double *params, chessfad_stream_t stream)
{
    return launch(fn, nullptr, true, n, batch, x, v, out, params, reinterpret_cast<cudaStream_t>(stream));
}

CHESSFAD_API int chessfad_user_hessian(chessfad_user_fn *fn, int n, long long batch, const void *x, void *H,
                                       const double *params, chessfad_stream_t stream)
{
    return launch(fn, nullptr, false, n, batch, x, nullptr, H, params, reinterpret_cast<cudaStream_t>(stream));
}

CHESSFAD_API int chessfad_user_hvp_config(chessfad_user_fn *fn, int n, long long batch, const chessfad_config *cfg,
                                          const void *x, const void *v, void *out, const double *params,
                                          chessfad_stream_t stream)
{
    return launch(fn, cfg, true, n, batch, x, v, out, params, reinterpret_cast<cudaStream_t>(stream));
}

CHESSFAD_API int chessfad_user_hessian_config(chessfad_user_fn *fn, int n, long long batch, const chessfad_config *cfg,
                                              const void *x, void *H, const double *params, chessfad_stream_t stream)
{
    return launch(fn, cfg, false, n, batch, x, nullptr, H, params, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
