// host_pipeline.cu -- H v for host-resident inputs and outputs, with the
// host-to-device copies, the sweeps and the device-to-host copies of
// consecutive slices of the batch overlapped.
//
// Points are independent (Sec. VI, L0), so the batch can be cut into slices
// that move through three stages: copy x and v in (copy engine), run the
// sweep kernel (SMs), copy the result out (the other copy engine).  Slice k's
// sweep overlaps slice k+1's input copy and slice k-1's output copy; sweeps
// alternate between two compute streams so the tail wave of one slice's
// kernel overlaps the start of the next.  Every internal stream first waits
// for the caller's stream, and the caller's stream finally waits for every
// internal stream, so the call behaves as one stream-ordered operation on the
// caller's stream (and can be captured into a CUDA graph from it).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <vector>

#include "../../include/chessfad.h"

namespace {

constexpr int kMaxSlices = 64;

struct Pipe {
    std::mutex mu;  // one enqueue sequence at a time per device (shared events)
    cudaStream_t h2d = nullptr, d2h = nullptr, comp[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev;  // start, 4 joins, then in/out per slice
};

std::mutex g_mu;
std::map<int, Pipe *> g_pipes;

// The per-device streams and events, created on first use with the device
// current; kept until the process exits.
Pipe *pipe_for(int dev)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_pipes.find(dev);
    if (it != g_pipes.end()) return it->second;
    auto *p = new Pipe;
    bool ok = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->comp[0], cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->comp[1], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < 5 + 2 * kMaxSlices; ++k) {
        cudaEvent_t e;
        ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) p->ev.push_back(e);
    }
    if (!ok) {
        cudaGetLastError();
        return nullptr;  // the partial Pipe is leaked deliberately: the device is unusable anyway
    }
    g_pipes[dev] = p;
    return p;
}

}  // namespace

extern "C" {

CHESSFAD_API int chessfad_hvp_host(int fn, int n, long long batch, int csize, const void *x_host,
                                   const void *v_host, void *out_host, void *x_dev, void *v_dev, void *out_dev,
                                   const chessfad_fp_params *params, int prec, int slices, chessfad_stream_t stream)
{
    // Every argument check of chessfad_hvp, without launching (batch 0).
    int st = chessfad_hvp(fn, n, 0, csize, nullptr, nullptr, nullptr, params, prec, stream);
    if (st != CHESSFAD_SUCCESS) return st;
    if (batch < 0) return CHESSFAD_ERR_BATCH;
    if (slices < 0 || slices > kMaxSlices) return CHESSFAD_ERR_CONFIG;
    if (batch == 0) return CHESSFAD_SUCCESS;
    if (!x_host || !v_host || !out_host || !x_dev || !v_dev || !out_dev) return CHESSFAD_ERR_NULL;
    int S = slices == 0 ? 8 : slices;
    if (S > batch) S = (int)batch;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    Pipe *p = pipe_for(dev);
    if (!p) return CHESSFAD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(p->mu);
    const cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    const size_t elem = (prec == CHESSFAD_FP64) ? sizeof(double) : sizeof(float);
    const cudaStream_t internal[4] = {p->h2d, p->comp[0], p->comp[1], p->d2h};
    cudaEvent_t *ev = p->ev.data();
    bool ok = cudaEventRecord(ev[0], caller) == cudaSuccess;
    for (cudaStream_t s : internal) ok = ok && cudaStreamWaitEvent(s, ev[0], 0) == cudaSuccess;
    for (int k = 0; ok && k < S; ++k) {
        const long long p0 = batch * k / S, p1 = batch * (k + 1) / S;
        const size_t off = (size_t)p0 * n * elem, bytes = (size_t)(p1 - p0) * n * elem;
        cudaEvent_t ein = ev[5 + 2 * k], eout = ev[6 + 2 * k];
        const cudaStream_t cs = p->comp[k & 1];
        ok = cudaMemcpyAsync(static_cast<char *>(x_dev) + off, static_cast<const char *>(x_host) + off, bytes,
                             cudaMemcpyHostToDevice, p->h2d) == cudaSuccess &&
             cudaMemcpyAsync(static_cast<char *>(v_dev) + off, static_cast<const char *>(v_host) + off, bytes,
                             cudaMemcpyHostToDevice, p->h2d) == cudaSuccess &&
             cudaEventRecord(ein, p->h2d) == cudaSuccess && cudaStreamWaitEvent(cs, ein, 0) == cudaSuccess;
        if (!ok) break;
        st = chessfad_hvp(fn, n, p1 - p0, csize, static_cast<char *>(x_dev) + off, static_cast<char *>(v_dev) + off,
                          static_cast<char *>(out_dev) + off, params, prec, reinterpret_cast<chessfad_stream_t>(cs));
        if (st != CHESSFAD_SUCCESS) break;
        ok = cudaEventRecord(eout, cs) == cudaSuccess && cudaStreamWaitEvent(p->d2h, eout, 0) == cudaSuccess &&
             cudaMemcpyAsync(static_cast<char *>(out_host) + off, static_cast<char *>(out_dev) + off, bytes,
                             cudaMemcpyDeviceToHost, p->d2h) == cudaSuccess;
    }
    // Join every internal stream back into the caller's stream, also after a
    // failure, so that no internal work is left unordered.
    for (int j = 0; j < 4; ++j) {
        const bool joined = cudaEventRecord(ev[1 + j], internal[j]) == cudaSuccess &&
                            cudaStreamWaitEvent(caller, ev[1 + j], 0) == cudaSuccess;
        ok = ok && joined;
    }
    if (st != CHESSFAD_SUCCESS) return st;
    return ok ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

}  // extern "C"
