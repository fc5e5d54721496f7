// ft_tune.cu -- ft_autotune: picks the launch shapes of the grid-stride kernels
// (canonical clip, column parity fill, PPIC accumulation, CSF dense pass), the
// segment count of the binning's scans, and
// the register/occupancy variant and cell schedule of the PPIC accumulation for the workload
// on a workspace, by timing each step with CUDA events, one parameter at a
// time, and installs the fastest.  The results of the steps do not depend on
// these choices; only their speed does.
#include <algorithm>
#include <vector>

#include "ft_internal.cuh"

namespace {

struct Buffers {
    double* alpha = nullptr;
    double* force = nullptr;
    double* kappa = nullptr;
    double* normal = nullptr;
    unsigned* keys = nullptr;
    int8_t* status = nullptr;
    void release() {
        void* p[] = {alpha, force, kappa, normal, keys, status};
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

// one pass of bin + alpha + PPIC + CSF; ms[4] receives each step's event time
struct Stepper {
    ft_workspace* ws;
    const ft_front* f;
    const ft_params* p;
    cudaStream_t s;
    Buffers b;
    cudaEvent_t ev[5];

    int run(float ms[4]) {
        int r = FT_OK;
        cudaEventRecord(ev[0], s);
        r = ws->batch ? front_bin_batch(ws, p, s) : front_bin(ws, f, p, s);
        cudaEventRecord(ev[1], s);
        if (r == FT_OK) r = ws->batch ? front_volume_fraction_batch(ws, s) : front_volume_fraction(ws, b.alpha, s);
        cudaEventRecord(ev[2], s);
        if (r == FT_OK)
            r = front_curvature_ppic(ws, p, ws->max_cells, b.keys, b.kappa, b.normal, nullptr, b.status, s);
        cudaEventRecord(ev[3], s);
        if (r == FT_OK)
            r = ws->batch ? front_csf_force_batch(ws, p, b.kappa, b.normal, s)
                          : front_csf_force(ws, p, b.alpha, b.kappa, b.normal, b.force, s);
        cudaEventRecord(ev[4], s);
        if (r != FT_OK) return r;
        if (cudaEventSynchronize(ev[4]) != cudaSuccess) return FT_ERR_CUDA;
        for (int i = 0; i < 4; i++) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        return FT_OK;
    }

    // median over `reps` runs (after one warm-up) of step `which` (-1: all four)
    int time(int which, int reps, double* out) {
        float ms[4];
        int r = run(ms);
        if (r != FT_OK) return r;
        std::vector<double> t;
        for (int i = 0; i < reps; i++) {
            r = run(ms);
            if (r != FT_OK) return r;
            t.push_back(which < 0 ? (double)ms[0] + ms[1] + ms[2] + ms[3] : (double)ms[which]);
        }
        std::sort(t.begin(), t.end());
        *out = t[t.size() / 2];
        return FT_OK;
    }
};

}  // namespace

extern "C" int ft_autotune(ft_workspace* ws, const ft_front* f, const ft_params* p, int32_t reps, ft_tuning* best,
                           void* stream) {
    if (!ws || !p || !best || reps < 1 || reps > 1000) return FT_ERR_ARG;
    if (ws->batch ? ws->nf < 1 : f == nullptr) return ws->batch ? FT_ERR_STATE : FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    Stepper st{ws, f, p, reinterpret_cast<cudaStream_t>(stream), Buffers{}, {}};
    const size_t Mx = (size_t)ws->max_cells;
    cudaError_t e = cudaSuccess;
    if (!ws->batch) {
        e = e ? e : cudaMalloc(&st.b.alpha, sizeof(double) * (size_t)ws->ncells);
        e = e ? e : cudaMalloc(&st.b.force, 3 * sizeof(double) * (size_t)ws->ncells);
    }
    e = e ? e : cudaMalloc(&st.b.kappa, sizeof(double) * Mx);
    e = e ? e : cudaMalloc(&st.b.normal, 3 * sizeof(double) * Mx);
    e = e ? e : cudaMalloc(&st.b.keys, sizeof(unsigned) * Mx);
    e = e ? e : cudaMalloc(&st.b.status, Mx);
    int created = 0;
    for (; e == cudaSuccess && created < 5; created++) e = cudaEventCreate(&st.ev[created]);
    int r = (e == cudaSuccess) ? FT_OK : FT_ERR_ALLOC;

    // the workload's needs, with the current shapes
    float ms[4];
    if (r == FT_OK) r = st.run(ms);
    ft_counters c = {};
    if (r == FT_OK && cudaMemcpy(&c, ws->ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) r = FT_ERR_CUDA;
    if (r == FT_OK && (c.status & FT_ST_CAPACITY)) r = FT_ERR_CAPACITY;

    // coordinate search: each step's time depends only on its own kernel's shape
    struct Knob {
        int* v;
        int step;
        std::vector<int> cand;
    };
    std::vector<int> segs;
    for (int g : {16, 32, 64, 96, 128, ws->grid_blocks})
        if (g <= ws->grid_blocks && (segs.empty() || segs.back() != g)) segs.push_back(g);
    Knob knobs[7] = {{&ws->tune.seg_blocks, 0, segs},
                     {&ws->tune.clip_bps, 0, {2, 3, 4, 6, 9, 12}},
                     {&ws->tune.fill_bps, 1, {2, 4, 8, 16}},
                     {&ws->tune.ppic_dynamic, 2, {0, 1}},
                     {&ws->tune.ppic_min_blocks, 2, {4, 6}},
                     {&ws->tune.ppic_bps, 2, {2, 3, 4, 6, 8}},
                     {&ws->tune.csf_bps, 3, {4, 8, 16, 32}}};
    for (int k = 0; k < 7 && r == FT_OK; k++) {
        Knob& K = knobs[k];
        int bv = *K.v;
        double bt = 1e30;
        for (int v : K.cand) {
            *K.v = v;
            double t;
            r = st.time(K.step, reps, &t);
            if (r != FT_OK) break;
            if (t < bt) {
                bt = t;
                bv = v;
            }
        }
        *K.v = bv;
    }
    double total = 0.0;
    if (r == FT_OK) r = st.time(-1, reps, &total);
    if (r == FT_OK) {
        ft_get_tuning(ws, best);
        best->cand_need = c.C_need;
        best->cells_need = c.M;
        best->fit_pairs = c.fit_pairs;
        best->step_ms = total;
    }
    // the status bits of the tuning runs are not the caller's
    cudaMemset(&ws->ctr->status, 0, sizeof(unsigned));
    if (ws->batch && ws->nf > 0) cudaMemset(ws->fstatus, 0, sizeof(unsigned) * ws->nf);
    cudaDeviceSynchronize();
    for (int i = 0; i < created; i++) cudaEventDestroy(st.ev[i]);
    st.b.release();
    return r;
}
