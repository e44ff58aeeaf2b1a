// batch.cu -- many independent detector instances (cells, resource blocks) of uneven size in one
// CUDA graph: apsm_batch_create records every instance's training and detection on parallel
// graph branches (longest instances first, each on the currently least-loaded branch), so one
// graph launch replays the whole batch with the branches running concurrently on the GPU.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "apsm_common.cuh"

struct apsm_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t n = 0;
};

namespace {

// Rough work of one instance (pair evaluations), used only to order and balance the branches.
double instance_work(const apsm_instance &x) {
    const double D = x.p.dict_cap, P = x.P, N = x.N;
    const double per_pair = 4.0 * x.p.M + 4.0 * x.p.K + 3.0;
    return per_pair * (N * std::min(D, P) + 0.5 * P * std::min(D, P)) + 2.0 * P * x.p.window * 400.0;
}

}  // namespace

extern "C" {

apsm_status apsm_batch_create(const apsm_instance *inst, int32_t n, int32_t lanes, apsm_batch *out) {
    if (!inst || n < 1 || !out || lanes < 1 || lanes > 64) return APSM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {  // every instance checked before anything is recorded
        const apsm_instance &x = inst[i];
        size_t need = 0;
        apsm_status s = apsm_train_workspace_bytes(&x.p, x.P, &need);
        if (s != APSM_OK) return s;
        if (x.N < 0 || (x.N > 0 && (!x.rx || !x.soft))) return APSM_ERR_INVALID_ARG;
        if (x.P > 0 && (!x.rx_pilot || !x.sym_pilot)) return APSM_ERR_INVALID_ARG;
        if (need > 0 && (!x.workspace || x.workspace_bytes < need)) return APSM_ERR_WORKSPACE;
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return instance_work(inst[a]) > instance_work(inst[b]); });
    lanes = std::min(lanes, n);

    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> ls(lanes, nullptr);
    std::vector<cudaEvent_t> done(lanes, nullptr);
    cudaEvent_t fork = nullptr;
    apsm_status st = APSM_OK;
    auto cleanup = [&]() {
        for (auto e : done)
            if (e) cudaEventDestroy(e);
        for (auto s : ls)
            if (s) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        if (origin) cudaStreamDestroy(origin);
    };
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
        cleanup();
        return APSM_ERR_CUDA;
    }
    for (int l = 0; l < lanes; ++l)
        if (cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[l], cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return APSM_ERR_CUDA;
        }
    apsm_batch_s *b = new (std::nothrow) apsm_batch_s();
    if (!b) {
        cleanup();
        return APSM_ERR_CUDA;
    }
    if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        delete b;
        cleanup();
        return APSM_ERR_CUDA;
    }
    cudaEventRecord(fork, origin);
    std::vector<double> load(lanes, 0.0);
    for (int l = 0; l < lanes; ++l) cudaStreamWaitEvent(ls[l], fork, 0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += instance_work(inst[i]);
        const apsm_instance &x = inst[i];
        st = apsm_train(&x.p, x.rx_pilot, x.sym_pilot, x.P, nullptr, &x.st, x.workspace, x.workspace_bytes,
                        nullptr, ls[l]);
        if (st == APSM_OK && x.N > 0) st = apsm_detect(&x.p, &x.st, x.rx, x.N, x.soft, x.hard, ls[l]);
        if (st != APSM_OK) break;
    }
    for (int l = 0; l < lanes; ++l) {
        cudaEventRecord(done[l], ls[l]);
        cudaStreamWaitEvent(origin, done[l], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
    if (st == APSM_OK && (ce != cudaSuccess || !graph)) st = APSM_ERR_CUDA;
    if (st == APSM_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) st = APSM_ERR_CUDA;
    cleanup();
    if (st != APSM_OK) {
        if (graph) cudaGraphDestroy(graph);
        delete b;
        cudaGetLastError();
        return st;
    }
    b->graph = graph;
    b->n = n;
    *out = b;
    return APSM_OK;
}

apsm_status apsm_batch_launch(apsm_batch b, void *stream) {
    if (!b || !b->exec) return APSM_ERR_INVALID_ARG;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? APSM_OK : APSM_ERR_CUDA;
}

apsm_status apsm_batch_destroy(apsm_batch b) {
    if (!b) return APSM_ERR_INVALID_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return APSM_OK;
}

}  // extern "C"
