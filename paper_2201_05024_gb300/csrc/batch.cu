// batch.cu -- many independent detector instances (cells, resource blocks) of uneven antenna
// count, user count, dictionary size and data length, trained and detected by one CUDA graph.
//
// Phase 1, training: every instance's training chain (apsm_train) is recorded on one of up to
// 64 parallel graph branches, longest instances first, each onto the currently least-loaded
// branch; the branches run concurrently on the GPU.
// Phase 2, detection: the instances are grouped by class (antenna count, user bucket).  Each
// class is one persistent launch of the batched tensor-core detection kernel: its CTAs take
// (instance, 128-query tile) work items from a device counter, listed longest instance first,
// until the list is exhausted (detect_tc_batch.cuh).  The counters are reset by memset nodes of
// the same graph.  Instances outside the batched kernel's range (BF16/FP16, 64 antennas, a class
// the launch-choice table gives to the FMA engine, larger-than-QPSK labels) are detected by
// apsm_detect on their branch right after their training.
// The work lists live in a caller-provided device workspace, written once at creation.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "apsm_common.cuh"
#include "detect_tc_batch.cuh"

namespace apsm {
TcBatchLauncher detect_tc_batch_launcher(int M, int K, int *ctas_per_sm);  // detect_dispatch.cu
bool tune_forces_ffma(int M, int K, int dtype);                           // apsm_api.cu
}  // namespace apsm

using namespace apsm;

struct apsm_batch_s {
    cudaGraphExec_t exec = nullptr;         // both phases
    cudaGraphExec_t exec_detect = nullptr;  // the persistent detection phase alone
    cudaGraph_t graph = nullptr, graph_detect = nullptr;
    int32_t n = 0, n_classes = 0, n_batched = 0;
};

namespace {

// Rough work of one instance (pair evaluations), used only to order and balance.
double instance_work(const apsm_instance &x) {
    const double D = x.p.dict_cap, P = x.P, N = x.N;
    const double per_pair = 4.0 * x.p.M + 4.0 * x.p.K + 3.0;
    return per_pair * (N * std::min(D, P) + 0.5 * P * std::min(D, P)) + 2.0 * P * x.p.window * 400.0;
}

// The batched kernel covers FP32 (TF32 x3 Gram) up to 32 antennas with QPSK decisions.
bool batched_detect(const apsm_instance &x) {
    const int mod = x.p.modulation == 0 ? 2 : x.p.modulation;
    int ctas = 0;
    return x.N > 0 && x.p.dtype == APSM_FP32 && x.p.M <= 32 && (mod == 2 || x.hard == nullptr) &&
           !tune_forces_ffma(x.p.M, x.p.K, x.p.dtype) && detect_tc_batch_launcher(x.p.M, x.p.K, &ctas) != nullptr;
}

struct BatchPlan {
    struct Class {
        int M, KB;
        std::vector<int> inst;  // instances, longest first
        size_t items = 0;
    };
    std::vector<Class> classes;
    size_t counters = 0, jobs = 0, items = 0, total = 0;
};

int bucket_of(int K) {
    static const int kB[] = {2, 4, 6, 8, 12, 16};
    for (int b : kB)
        if (b >= K) return b;
    return 0;
}

BatchPlan plan_batch(const apsm_instance *inst, int n) {
    BatchPlan pl;
    for (int i = 0; i < n; ++i) {
        if (!batched_detect(inst[i])) continue;
        const int M = inst[i].p.M, KB = bucket_of(inst[i].p.K);
        auto it = std::find_if(pl.classes.begin(), pl.classes.end(),
                               [&](const BatchPlan::Class &c) { return c.M == M && c.KB == KB; });
        if (it == pl.classes.end()) {
            pl.classes.push_back(BatchPlan::Class{M, KB, {}, 0});
            it = pl.classes.end() - 1;
        }
        it->inst.push_back(i);
        it->items += (size_t)(inst[i].N + kTcRows - 1) / kTcRows;
    }
    size_t n_jobs = 0, n_items = 0;
    for (auto &c : pl.classes) {
        // longest instance first: the most entry tiles per item, then the most items
        std::stable_sort(c.inst.begin(), c.inst.end(), [&](int a, int b) {
            const int ta = (inst[a].p.dict_cap + kTcEntries - 1) / kTcEntries;
            const int tb = (inst[b].p.dict_cap + kTcEntries - 1) / kTcEntries;
            return ta != tb ? ta > tb : inst[a].N > inst[b].N;
        });
        n_jobs += c.inst.size();
        n_items += c.items;
    }
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    pl.counters = 0;
    pl.jobs = al(sizeof(int) * pl.classes.size());
    pl.items = al(pl.jobs + sizeof(TcArgs) * n_jobs);
    pl.total = pl.classes.empty() ? 0 : al(pl.items + sizeof(int2) * n_items);
    return pl;
}

apsm_status validate(const apsm_instance *inst, int32_t n) {
    for (int i = 0; i < n; ++i) {
        const apsm_instance &x = inst[i];
        size_t need = 0;
        apsm_status s = apsm_train_workspace_bytes(&x.p, x.P, &need);
        if (s != APSM_OK) return s;
        if (x.N < 0 || (x.N > 0 && (!x.rx || !x.soft))) return APSM_ERR_INVALID_ARG;
        if (x.P > 0 && (!x.rx_pilot || !x.sym_pilot)) return APSM_ERR_INVALID_ARG;
        if (need > 0 && (!x.workspace || x.workspace_bytes < need)) return APSM_ERR_WORKSPACE;
    }
    return APSM_OK;
}

}  // namespace

extern "C" {

apsm_status apsm_batch_workspace_bytes(const apsm_instance *inst, int32_t n, size_t *bytes) {
    if (!inst || n < 1 || !bytes) return APSM_ERR_INVALID_ARG;
    apsm_status s = validate(inst, n);
    if (s != APSM_OK) return s;
    *bytes = plan_batch(inst, n).total;
    return APSM_OK;
}

apsm_status apsm_batch_create(const apsm_instance *inst, int32_t n, int32_t lanes, void *workspace,
                              size_t workspace_bytes, apsm_batch *out) {
    if (!inst || n < 1 || !out || lanes < 1 || lanes > 64) return APSM_ERR_INVALID_ARG;
    *out = nullptr;
    apsm_status s = validate(inst, n);  // every instance checked before anything is recorded
    if (s != APSM_OK) return s;
    const BatchPlan pl = plan_batch(inst, n);
    if (pl.total > 0 && (!workspace || workspace_bytes < pl.total)) return APSM_ERR_WORKSPACE;
    if (pl.total > 0 && (reinterpret_cast<uintptr_t>(workspace) & 255)) return APSM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return APSM_ERR_CUDA;
    }

    // ---- the work lists (descriptors as apsm_detect builds them), written once ----------------
    unsigned char *wsb = static_cast<unsigned char *>(workspace);
    std::vector<TcArgs> jobs;
    std::vector<int2> items;
    std::vector<size_t> job0, item0;  // first job / item of each class
    for (const auto &c : pl.classes) {
        job0.push_back(jobs.size());
        item0.push_back(items.size());
        for (int i : c.inst) {
            const apsm_instance &x = inst[i];
            TcArgs ta{};
            ta.rx = reinterpret_cast<const float2 *>(x.rx);
            ta.N = x.N;
            ta.dict = reinterpret_cast<const float2 *>(x.st.dict);
            ta.dict_norm = x.st.dict_norm;
            ta.gamma = x.st.gamma;
            ta.clin = reinterpret_cast<const float2 *>(x.st.clin);
            ta.meta = x.st.meta;
            ta.n_entries = x.p.dict_cap;
            ta.K = x.p.K;
            ta.half_fmt = 0;
            ta.k2 = kLog2e / (2.f * x.p.sigma * x.p.sigma);
            ta.wL = x.p.w_L;
            ta.wG = 1.f - x.p.w_L;
            ta.soft = reinterpret_cast<float2 *>(x.soft);
            ta.hard = x.hard;
            ta.status = x.st.meta + 3;
            const int j = (int)(jobs.size() - job0.back());
            jobs.push_back(ta);
            for (int q = 0; q < x.N; q += kTcRows) items.push_back(make_int2(j, q));
        }
    }
    if (pl.total > 0) {
        if (cudaMemset(wsb + pl.counters, 0, sizeof(int) * pl.classes.size()) != cudaSuccess ||
            cudaMemcpy(wsb + pl.jobs, jobs.data(), sizeof(TcArgs) * jobs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(wsb + pl.items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return APSM_ERR_CUDA;
        }
    }
    // the persistent detection launches of every class, recorded on `strm`
    auto record_detect = [&](cudaStream_t strm) -> apsm_status {
        for (size_t c = 0; c < pl.classes.size(); ++c) {
            int ctas = 0;
            const TcBatchLauncher fn = detect_tc_batch_launcher(pl.classes[c].M, pl.classes[c].KB, &ctas);
            int *counter = reinterpret_cast<int *>(wsb + pl.counters) + c;
            TcBatchArgs ba{};
            ba.jobs = reinterpret_cast<const TcArgs *>(wsb + pl.jobs) + job0[c];
            ba.items = reinterpret_cast<const int2 *>(wsb + pl.items) + item0[c];
            ba.n_items = (int)pl.classes[c].items;
            ba.counter = counter;
            ba.half_fmt = 0;
            const int grid = (int)std::min<size_t>(pl.classes[c].items, (size_t)sms * std::max(ctas, 1));
            if (!fn || cudaMemsetAsync(counter, 0, sizeof(int), strm) != cudaSuccess ||
                fn(ba, grid, strm) != cudaSuccess)
                return APSM_ERR_CUDA;
        }
        return APSM_OK;
    };

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
    // graph 1: training on parallel branches (plus the detection of instances outside the
    // batched kernel), then the persistent detection launches
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
        if (st == APSM_OK && x.N > 0 && !batched_detect(x))
            st = apsm_detect(&x.p, &x.st, x.rx, x.N, x.soft, x.hard, ls[l]);
        if (st != APSM_OK) break;
    }
    for (int l = 0; l < lanes; ++l) {
        cudaEventRecord(done[l], ls[l]);
        cudaStreamWaitEvent(origin, done[l], 0);
    }
    if (st == APSM_OK) st = record_detect(origin);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(origin, &graph);
    if (st == APSM_OK && (ce != cudaSuccess || !graph)) st = APSM_ERR_CUDA;
    if (st == APSM_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) st = APSM_ERR_CUDA;
    b->graph = graph;
    // graph 2: the detection phase alone (to time it)
    if (st == APSM_OK && !pl.classes.empty()) {
        cudaGraph_t g2 = nullptr;
        if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = APSM_ERR_CUDA;
        if (st == APSM_OK) st = record_detect(origin);
        ce = cudaStreamEndCapture(origin, &g2);
        if (st == APSM_OK && (ce != cudaSuccess || !g2)) st = APSM_ERR_CUDA;
        if (st == APSM_OK && cudaGraphInstantiate(&b->exec_detect, g2, 0) != cudaSuccess) st = APSM_ERR_CUDA;
        b->graph_detect = g2;
    }
    cleanup();
    if (st != APSM_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->exec_detect) cudaGraphExecDestroy(b->exec_detect);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->graph_detect) cudaGraphDestroy(b->graph_detect);
        delete b;
        cudaGetLastError();
        return st;
    }
    b->n = n;
    b->n_classes = (int32_t)pl.classes.size();
    for (const auto &c : pl.classes) b->n_batched += (int32_t)c.inst.size();
    *out = b;
    return APSM_OK;
}

apsm_status apsm_batch_launch(apsm_batch b, void *stream) {
    if (!b || !b->exec) return APSM_ERR_INVALID_ARG;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? APSM_OK : APSM_ERR_CUDA;
}

apsm_status apsm_batch_launch_detect(apsm_batch b, void *stream) {
    if (!b) return APSM_ERR_INVALID_ARG;
    if (!b->exec_detect) return APSM_OK;  // no instance in the batched kernel's range
    return cudaGraphLaunch(b->exec_detect, static_cast<cudaStream_t>(stream)) == cudaSuccess ? APSM_OK
                                                                                             : APSM_ERR_CUDA;
}

apsm_status apsm_batch_info(apsm_batch b, int32_t *n_classes, int32_t *n_batched) {
    if (!b || !n_classes || !n_batched) return APSM_ERR_INVALID_ARG;
    *n_classes = b->n_classes;
    *n_batched = b->n_batched;
    return APSM_OK;
}

apsm_status apsm_batch_destroy(apsm_batch b) {
    if (!b) return APSM_ERR_INVALID_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->exec_detect) cudaGraphExecDestroy(b->exec_detect);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->graph_detect) cudaGraphDestroy(b->graph_detect);
    delete b;
    return APSM_OK;
}

}  // extern "C"
