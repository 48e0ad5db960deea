// A serving loop for merge-tree requests on one GPU (continuous batching).
//
// The server owns one device allocation (its HBM budget) carved by a first-fit
// allocator, and max_slots CUDA streams. A worker thread admits pending
// requests, in arrival order but skipping any that do not fit yet, as soon as
// a slot and enough of the budget are free; admitted requests run on their own
// streams, so requests that arrive while others are on the GPU overlap with
// them. For each request the field is copied in, the triplet tree is built,
// the pairs are compacted and the labels at the request's threshold are
// computed (the same library calls as a single request), and the results are
// copied back. The pair count is read back first (stage 1) so that stage 2
// copies exactly the pairs that exist. Results do not depend on what else is
// running: every request works on its own buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mt.h"
#include "mt_internal.h"

namespace mt {

mt_status status_from_bits(uint32_t bits);  // mt_api.cu

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over one device range; host-side bookkeeping only.
class Pool {
  public:
    void init(char *base, size_t bytes)
    {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
    }
    // returns the offset or SIZE_MAX
    size_t alloc(size_t bytes)
    {
        bytes = al256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = al256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *base() const { return base_; }

  private:
    char *base_ = nullptr;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Request {
    uint64_t ticket;
    const float *h_f;
    mt_grid g;
    float t;
    uint32_t *h_pairs;
    uint64_t pair_cap;
    uint32_t *h_labels;
    double t_submit;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev1 = nullptr, ev2 = nullptr;
    int stage = 0;  // 0 free, 1 computing, 2 copying pairs
    mt_status keep = MT_OK;  // status decided at the end of stage 1
    Request req;
    size_t off = 0, bytes = 0;
    uint64_t *h_meta = nullptr;  // pinned: [0] npairs [1] roots [2] root [3] status bits
    double t_admit = 0;
    // device views
    float *f = nullptr;
    uint64_t *W = nullptr;
    uint32_t *labels = nullptr, *pairs = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint64_t dev_cap = 0;
};

size_t request_bytes(uint64_t n, size_t ws_bytes, uint64_t cap)
{
    return al256(4 * n) + al256(8 * n) + al256(4 * n) + al256(8 * cap) + al256(ws_bytes);
}

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0;
    char *dbase = nullptr;
    Pool pool;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::map<uint64_t, mt_result> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    void run();
    bool admit(Slot &s, const Request &r);
    void finish(Slot &s, mt_status st);
};

bool Server::admit(Slot &s, const Request &r)
{
    const uint64_t n = (uint64_t)r.g.nx * r.g.ny * r.g.nz;
    mt_grid g = r.g;
    const size_t wsb = mt_workspace_bytes(g);
    const uint64_t cap = n / 2 + 1;  // minima are never adjacent: fewer than n/2 pairs
    const size_t bytes = request_bytes(n, wsb, cap);
    const size_t off = pool.alloc(bytes);
    if (off == SIZE_MAX) return false;
    char *p = pool.base() + off;
    s.off = off;
    s.bytes = bytes;
    s.f = reinterpret_cast<float *>(p);
    p += al256(4 * n);
    s.W = reinterpret_cast<uint64_t *>(p);
    p += al256(8 * n);
    s.labels = reinterpret_cast<uint32_t *>(p);
    p += al256(4 * n);
    s.pairs = reinterpret_cast<uint32_t *>(p);
    p += al256(8 * cap);
    s.ws = p;
    s.ws_bytes = wsb;
    s.dev_cap = cap;
    s.req = r;
    s.t_admit = now_s();
    s.stage = 1;
    s.keep = MT_OK;
    std::memset(s.h_meta, 0, 4 * sizeof(uint64_t));
    cudaStream_t st = s.st;
    bool ok = cudaMemcpyAsync(s.f, r.h_f, 4 * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && mt_build_triplets(s.f, g, s.W, s.ws, s.ws_bytes, st) == MT_OK;
    Workspace ws;
    ok = ok && carve_workspace(s.ws, s.ws_bytes, n, ws);
    ok = ok && launch_pairs(s.W, n, s.pairs, cap, ws, st) == cudaSuccess;
    ok = ok && mt_components_at(s.f, s.W, g, r.t, s.labels, s.ws, s.ws_bytes, st) == MT_OK;
    ok = ok && cudaMemcpyAsync(s.h_meta, ws.meta, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(s.h_meta + 3, ws.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (r.h_labels)
        ok = ok && cudaMemcpyAsync(r.h_labels, s.labels, 4 * n, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaEventRecord(s.ev1, st) == cudaSuccess;
    if (!ok) {
        cudaStreamSynchronize(st);
        finish(s, MT_ERR_CUDA);
    }
    return true;
}

void Server::finish(Slot &s, mt_status st)
{
    mt_result res;
    std::memset(&res, 0, sizeof(res));
    res.status = st;
    res.npairs = s.h_meta ? s.h_meta[0] : 0;
    res.root = (s.h_meta && s.h_meta[1] == 1) ? (uint32_t)s.h_meta[2] : 0xFFFFFFFFu;
    res.t_submit = s.req.t_submit;
    res.t_admit = s.t_admit;
    res.t_done = now_s();
    pool.release(s.off, s.bytes);
    s.stage = 0;
    done[s.req.ticket] = res;
    cv_done.notify_all();
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        bool progressed = false;
        // admit: arrival order, skipping requests that do not fit yet
        for (auto it = pending.begin(); it != pending.end();) {
            Slot *free_slot = nullptr;
            for (auto &s : slots)
                if (s.stage == 0) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot) break;
            if (admit(*free_slot, *it)) {
                it = pending.erase(it);
                progressed = true;
            } else {
                ++it;
            }
        }
        // advance in-flight requests
        for (auto &s : slots) {
            if (s.stage == 1 && cudaEventQuery(s.ev1) == cudaSuccess) {
                const uint32_t bits = (uint32_t)s.h_meta[3];
                mt_status st = bits ? status_from_bits(bits) : MT_OK;
                const uint64_t np = s.h_meta[0];
                if (st == MT_OK && s.h_meta[1] != 1) st = MT_ERR_INVALID;
                const uint64_t k = std::min(np, s.req.pair_cap);
                if (st == MT_OK && np > s.req.pair_cap) st = MT_ERR_CAPACITY;
                if ((st == MT_OK || st == MT_ERR_CAPACITY) && k && s.req.h_pairs) {
                    s.stage = 2;
                    s.keep = st;
                    if (cudaMemcpyAsync(s.req.h_pairs, s.pairs, 8 * k, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
                        cudaEventRecord(s.ev2, s.st) != cudaSuccess) {
                        cudaStreamSynchronize(s.st);
                        finish(s, MT_ERR_CUDA);
                    }
                } else {
                    finish(s, st);
                }
                progressed = true;
            } else if (s.stage == 2 && cudaEventQuery(s.ev2) == cudaSuccess) {
                finish(s, s.keep);
                progressed = true;
            }
        }
        bool busy = false;
        for (auto &s : slots) busy |= s.stage != 0;
        if (stop && !busy && pending.empty()) break;
        if (!progressed) {
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

}  // namespace mt

using namespace mt;

struct mt_server {
    Server s;
};

extern "C" {

mt_server *mt_server_create(size_t hbm_budget_bytes, int max_slots, int device)
{
    if (hbm_budget_bytes < (1u << 20) || max_slots < 1 || max_slots > 64) return nullptr;
    auto *srv = new mt_server();
    Server &S = srv->s;
    S.device = device;
    S.budget = hbm_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&S.dbase, hbm_budget_bytes) != cudaSuccess) {
        delete srv;
        return nullptr;
    }
    S.pool.init(S.dbase, hbm_budget_bytes);
    S.slots.resize(max_slots);
    for (auto &sl : S.slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev2, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.h_meta), 4 * sizeof(uint64_t), cudaHostAllocDefault) !=
                cudaSuccess) {
            mt_server_destroy(srv);
            return nullptr;
        }
    }
    S.worker = std::thread([&S] { S.run(); });
    return srv;
}

mt_status mt_server_submit(mt_server *srv, const float *h_f, mt_grid g, float t, uint32_t *h_pairs,
                           uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket)
{
    if (!srv || !h_f || !ticket || g.nx == 0 || g.ny == 0 || g.nz == 0 || t != t) return MT_ERR_INVALID;
    const uint64_t n = (uint64_t)g.nx * g.ny * g.nz;
    if (n >= 0xFFFFFFFFull) return MT_ERR_TOO_LARGE;
    Server &S = srv->s;
    if (request_bytes(n, mt_workspace_bytes(g), n / 2 + 1) > S.budget) return MT_ERR_NOMEM;
    std::lock_guard<std::mutex> lk(S.mu);
    Request r{S.next_ticket++, h_f, g, t, h_pairs, h_pairs ? pair_cap : 0, h_labels, now_s()};
    S.pending.push_back(r);
    *ticket = r.ticket;
    S.cv_work.notify_one();
    return MT_OK;
}

mt_status mt_server_poll(mt_server *srv, uint64_t ticket, mt_result *r)
{
    if (!srv || !r) return MT_ERR_INVALID;
    Server &S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.done.find(ticket);
    if (it == S.done.end()) return ticket && ticket < S.next_ticket ? MT_ERR_BUSY : MT_ERR_INVALID;
    *r = it->second;
    S.done.erase(it);
    return MT_OK;
}

mt_status mt_server_wait(mt_server *srv, uint64_t ticket, mt_result *r)
{
    if (!srv || !r) return MT_ERR_INVALID;
    Server &S = srv->s;
    std::unique_lock<std::mutex> lk(S.mu);
    if (!ticket || ticket >= S.next_ticket) return MT_ERR_INVALID;
    S.cv_done.wait(lk, [&] { return S.done.count(ticket) != 0; });
    *r = S.done[ticket];
    S.done.erase(ticket);
    return MT_OK;
}

void mt_server_destroy(mt_server *srv)
{
    if (!srv) return;
    Server &S = srv->s;
    if (S.worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.stop = true;
            S.cv_work.notify_one();
        }
        S.worker.join();
    }
    cudaSetDevice(S.device);
    for (auto &sl : S.slots) {
        if (sl.st) cudaStreamSynchronize(sl.st), cudaStreamDestroy(sl.st);
        if (sl.ev1) cudaEventDestroy(sl.ev1);
        if (sl.ev2) cudaEventDestroy(sl.ev2);
        if (sl.h_meta) cudaFreeHost(sl.h_meta);
    }
    if (S.dbase) cudaFree(S.dbase);
    delete srv;
}

}  // extern "C"
