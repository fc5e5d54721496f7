// ft_trace.cu -- per-kernel timing of the library's own launches (no
// counterpart in the paper): while a trace is open, every traced launch is
// bracketed by two CUDA events recorded on its own stream, so that a caller can
// read each kernel's device time (ft_trace_start / ft_trace_stop in front.h).
// Launches made during stream capture are never traced (an event record there
// would become part of the graph).
#include <string.h>

#include <mutex>
#include <vector>

#include "ft_internal.cuh"

namespace {

struct Slot {
    const char* name;
    cudaEvent_t e0, e1;
};

std::mutex g_mu;
bool g_on = false;           // guarded by g_mu; read without the lock as a hint
std::vector<Slot> g_slots;   // event pairs created by ft_trace_start
long long g_used = 0;        // slots taken by traced launches
long long g_dropped = 0;     // traced launches beyond the capacity

void free_slots() {
    for (Slot& s : g_slots) {
        cudaEventDestroy(s.e0);
        cudaEventDestroy(s.e1);
    }
    g_slots.clear();
    g_used = g_dropped = 0;
}

}  // namespace

namespace ft {

Trace::Trace(cudaStream_t s, const char* name) : slot_(-1), s_(s) {
    if (!__atomic_load_n(&g_on, __ATOMIC_ACQUIRE)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    if (g_used >= (long long)g_slots.size()) {
        g_dropped++;
        return;
    }
    slot_ = g_used++;
    g_slots[slot_].name = name;
    cudaEventRecord(g_slots[slot_].e0, s);
}

Trace::~Trace() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_slots[slot_].e1, s_);
}

}  // namespace ft

extern "C" {

int ft_trace_start(int64_t capacity) {
    if (capacity < 1 || capacity > (1 << 22)) return FT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_on) return FT_ERR_STATE;
    free_slots();
    g_slots.resize((size_t)capacity);
    for (long long i = 0; i < capacity; i++) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            g_slots.resize((size_t)i);  // the pairs created so far
            free_slots();
            return FT_ERR_CUDA;
        }
        g_slots[i] = Slot{nullptr, e0, e1};
    }
    __atomic_store_n(&g_on, true, __ATOMIC_RELEASE);
    return FT_OK;
}

int ft_trace_stop(int32_t max_kernels, char* names, int64_t* launches, double* total_ms, int32_t* n_kernels,
                  int64_t* dropped) {
    if (max_kernels < 0 || (max_kernels > 0 && (!names || !launches || !total_ms)) || !n_kernels)
        return FT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return FT_ERR_STATE;
    __atomic_store_n(&g_on, false, __ATOMIC_RELEASE);
    int nk = 0;
    int rc = FT_OK;
    for (long long i = 0; i < g_used; i++) {
        Slot& s = g_slots[i];
        if (cudaEventSynchronize(s.e1) != cudaSuccess) {
            rc = FT_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s.e0, s.e1) != cudaSuccess) {
            rc = FT_ERR_CUDA;
            break;
        }
        int k = 0;
        while (k < nk && strncmp(names + (size_t)k * FT_TRACE_NAME, s.name, FT_TRACE_NAME - 1) != 0) k++;
        if (k == nk) {
            if (nk == max_kernels) {
                rc = FT_ERR_CAPACITY;
                continue;
            }
            char* dst = names + (size_t)nk * FT_TRACE_NAME;
            strncpy(dst, s.name, FT_TRACE_NAME - 1);
            dst[FT_TRACE_NAME - 1] = 0;
            launches[nk] = 0;
            total_ms[nk] = 0.0;
            nk++;
        }
        launches[k]++;
        total_ms[k] += (double)ms;
    }
    *n_kernels = nk;
    if (dropped) *dropped = g_dropped;
    free_slots();
    return rc;
}

}  // extern "C"
