// Batched form: many independent TT-S_N problems of uneven sizes stepped
// together.  Each problem is a full handle (tt_create) on its own CUDA stream;
// a pool of host threads advances the problems concurrently, so the small
// per-problem kernels of different problems overlap on the GPU and each
// problem's rank decisions wait only for its own stream.  With captured steps
// (tt_batch_set_graph) a batch step is one launch of a graph that holds every
// problem's recorded step as a branch of its own.
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace ttsn;

struct tt_batch_ctx {
    int device = 0;
    std::vector<tt_handle> h;
    std::vector<cudaStream_t> streams;
    int threads = 1;
    bool graph = false;  // captured steps (tt_batch_set_graph)
    // all problems' captured steps as one graph (a branch per problem),
    // replayed on `origin` and ordered with the problems' streams by events
    cudaGraphExec_t bexec = nullptr;
    unsigned blaunches = 0;
    cudaStream_t origin = nullptr;
    std::vector<cudaEvent_t> evs;
    void drop_graph() {
        if (bexec) cudaGraphExecDestroy(bexec);
        bexec = nullptr;
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        evs.clear();
        if (origin) cudaStreamDestroy(origin);
        origin = nullptr;
    }
    ~tt_batch_ctx() {
        drop_graph();
        for (tt_handle x : h) tt_destroy(x);
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
    }
};

extern "C" {

tt_status tt_batch_create(const tt_problem_desc* descs, int count, int threads, tt_batch* out) {
    set_error("");
    if (!descs || !out || count <= 0) {
        set_error("tt_batch_create: need descs, out and count > 0");
        return TT_ERR_ARG;
    }
    *out = nullptr;
    tt_batch_ctx* b = new tt_batch_ctx();
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        set_error("tt_batch_create: no current device");
        return TT_ERR_CUDA;
    }
    // default: one host thread per hardware thread (on a 16-core host the
    // 64-problem workload measured 418 / 456 / 442 / 414 problem-steps/s with
    // 8 / 16 / 32 / 64 threads: more threads than cores only add contention)
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    b->threads = threads > 0 ? threads : std::min(count, hw);
    for (int i = 0; i < count; ++i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            set_error("tt_batch_create: stream creation failed");
            return TT_ERR_CUDA;
        }
        b->streams.push_back(s);
        tt_handle h = nullptr;
        tt_status st = tt_create(&descs[i], s, &h);
        if (st < 0) {
            std::string msg = std::string("tt_batch_create: problem ") + std::to_string(i) + ": " + tt_last_error();
            delete b;
            set_error(msg);
            return st;
        }
        b->h.push_back(h);
    }
    *out = b;
    return TT_OK;
}

tt_status tt_batch_step(tt_batch b, int nsteps, tt_step_info* infos) {
    set_error("");
    if (!b) {
        set_error("tt_batch_step: null batch");
        return TT_ERR_ARG;
    }
    const int n = (int)b->h.size();
    if (b->graph && nsteps > 0) {
        // one graph launch per batch step (every problem a branch of it), then
        // one wait per problem
        if (!b->bexec) {
            TT_TRY(graph_batch_build(b->h.data(), n, &b->bexec, &b->blaunches));
            if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) {
                b->drop_graph();
                set_error("tt_batch_step: stream creation failed");
                return TT_ERR_CUDA;
            }
            b->evs.assign(n + 1, nullptr);
            for (auto& e : b->evs)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                    b->drop_graph();
                    set_error("tt_batch_step: event creation failed");
                    return TT_ERR_CUDA;
                }
        }
        TT_TRY(graph_batch_launch(b->h.data(), n, b->bexec, b->blaunches, b->origin, b->evs.data(), nsteps));
        tt_status result = TT_OK;
        for (int i = 0; i < n; ++i) {
            tt_status st = graph_steps_end(b->h[i], infos ? &infos[i] : nullptr);
            if (st < 0) {
                std::string msg = std::string("problem ") + std::to_string(i) + ": " + tt_last_error();
                set_error(msg);
                return st;
            }
            if (st == TT_WARN_RANK_CAPPED) result = TT_WARN_RANK_CAPPED;
        }
        return result;
    }
    std::atomic<int> next{0};
    std::vector<tt_status> status(n, TT_OK);
    std::vector<std::string> errs(n);
    auto worker = [&]() {
        cudaSetDevice(b->device);
        for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
            status[i] = tt_sn_step_ex(b->h[i], nsteps, 0, nullptr, infos ? &infos[i] : nullptr);
            if (status[i] < 0) errs[i] = tt_last_error();
        }
    };
    const int nt = std::max(1, std::min(b->threads, n));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    tt_status result = TT_OK;
    for (int i = 0; i < n; ++i) {
        if (status[i] < 0) {
            set_error(std::string("problem ") + std::to_string(i) + ": " + errs[i]);
            return status[i];
        }
        if (status[i] == TT_WARN_RANK_CAPPED) result = TT_WARN_RANK_CAPPED;
    }
    return result;
}

tt_status tt_batch_size(tt_batch b, int* count) {
    if (!b || !count) {
        set_error("tt_batch_size: null argument");
        return TT_ERR_ARG;
    }
    *count = (int)b->h.size();
    return TT_OK;
}

tt_status tt_batch_handle(tt_batch b, int i, tt_handle* out) {
    if (!b || !out || i < 0 || i >= (int)b->h.size()) {
        set_error("tt_batch_handle: bad batch or index");
        return TT_ERR_ARG;
    }
    *out = b->h[i];
    return TT_OK;
}

tt_status tt_batch_sync(tt_batch b) {
    if (!b) {
        set_error("tt_batch_sync: null batch");
        return TT_ERR_ARG;
    }
    for (tt_handle h : b->h) TT_TRY(tt_sync(h));
    return TT_OK;
}

void tt_batch_destroy(tt_batch b) { delete b; }

tt_status tt_batch_set_graph(tt_batch b, int enable) {
    set_error("");
    if (!b) {
        set_error("tt_batch_set_graph: null batch");
        return TT_ERR_ARG;
    }
    if (enable) {
        for (size_t i = 0; i < b->h.size(); ++i) {
            tt_status st = tt_set_graph(b->h[i], 1);
            if (st < 0) {
                std::string msg = std::string("problem ") + std::to_string(i) + ": " + tt_last_error();
                for (size_t j = 0; j < i; ++j) tt_set_graph(b->h[j], 0);
                set_error(msg);
                return st;
            }
        }
    } else {
        for (tt_handle h : b->h) TT_TRY(tt_set_graph(h, 0));
    }
    if (!enable) b->drop_graph();
    b->graph = enable != 0;
    return TT_OK;
}

}  // extern "C"
