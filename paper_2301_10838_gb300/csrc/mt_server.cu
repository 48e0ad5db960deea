// A serving loop for merge-tree requests on one GPU (continuous batching).
//
// The server owns one device allocation (its HBM budget) carved by a first-fit
// allocator, and max_slots CUDA streams. A worker thread admits pending
// requests, in arrival order but skipping any that do not fit yet, as soon as
// a slot and enough of the budget are free; admitted requests run on their own
// streams, so requests that arrive while others are on the GPU overlap with
// them. A request that has been overtaken kMaxOvertakes times stops admission
// behind it until it fits, so a large request cannot be starved by a stream
// of small ones. For each request the field is copied in, the triplet tree is
// built, the pairs are compacted and the labels at the request's threshold
// are computed (the same library calls as a single request), and the results
// are copied back. The pair count is read back first (stage 1) so that stage
// 2 copies exactly the pairs that exist. Results do not depend on what else is
// running: every request works on its own buffers.
//
// Resident fields: a request submitted with a nonzero key keeps its field,
// its triplet tree and its pairs on the device after it completes. A later
// request with the same key only computes the labels at its own threshold
// (the tree and the pairs do not depend on it) and copies the stored pairs.
// Resident entries that no running request uses are evicted, least recently
// used first, when an admission needs their memory, or on request.
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
    uint64_t key;        // 0: a one-off request; else the resident field it builds or reuses
    uint32_t overtaken;  // requests admitted after this one arrived while it waited
};

// A field kept on the device with its tree and pairs (keyed requests).
struct Resident {
    mt_grid g{};
    size_t off = 0, bytes = 0;  // pool allocation: f, W, pairs
    float *f = nullptr;
    uint64_t *W = nullptr;
    uint32_t *pairs = nullptr;
    uint64_t npairs = 0, nroots = 0;
    uint32_t root = 0xFFFFFFFFu;
    bool ready = false;   // built; false while the building request runs
    bool evict = false;   // drop once no request uses it
    int users = 0;        // admitted requests that use it
    double last_use = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev1 = nullptr, ev2 = nullptr;
    int stage = 0;  // 0 free, 1 computing, 2 copying pairs
    mt_status keep = MT_OK;  // status decided at the end of stage 1
    Request req;
    size_t off = 0, bytes = 0;   // this request's own allocation
    uint64_t *h_meta = nullptr;  // pinned: [0] npairs [1] roots [2] root [3] status bits
    double t_admit = 0;
    bool builds = false;         // stage 1 builds the tree (else a resident tree is reused)
    // device views
    float *f = nullptr;
    uint64_t *W = nullptr;
    uint32_t *labels = nullptr, *pairs = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint64_t dev_cap = 0;
};

// Requests admitted behind a waiting one before it blocks admission.
constexpr uint32_t kMaxOvertakes = 8;

// Device bytes of a request: the part a resident entry keeps (field,
// triplets, pairs) and the part every request needs for itself (labels,
// workspace).
size_t kept_bytes(uint64_t n, uint64_t cap) { return al256(4 * n) + al256(8 * n) + al256(8 * cap); }
size_t own_bytes(uint64_t n, size_t ws_bytes) { return al256(4 * n) + al256(ws_bytes); }
size_t request_bytes(uint64_t n, size_t ws_bytes, uint64_t cap) { return kept_bytes(n, cap) + own_bytes(n, ws_bytes); }

bool same_grid(const mt_grid &a, const mt_grid &b) { return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz; }

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
    std::map<uint64_t, Resident> resident;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    enum Admit { kAdmitted, kNoRoom, kWait, kFailed };
    void run();
    Admit admit(Slot &s, const Request &r, mt_status &fail);
    size_t alloc_evicting(size_t bytes, uint64_t keep_key);
    void drop_resident(uint64_t key);
    void finish(Slot &s, mt_status st);
    void complete(const Request &r, mt_status st);
};

// Releases a resident entry's memory and forgets it.
void Server::drop_resident(uint64_t key)
{
    auto it = resident.find(key);
    if (it == resident.end()) return;
    pool.release(it->second.off, it->second.bytes);
    resident.erase(it);
}

// Allocates from the pool; when it is full, evicts idle resident entries
// (ready, no users), least recently used first, and tries again.
size_t Server::alloc_evicting(size_t bytes, uint64_t keep_key)
{
    for (;;) {
        const size_t off = pool.alloc(bytes);
        if (off != SIZE_MAX) return off;
        uint64_t victim = 0;
        double oldest = 0;
        for (auto &kv : resident) {
            const Resident &e = kv.second;
            if (kv.first == keep_key || !e.ready || e.users) continue;
            if (!victim || e.last_use < oldest) victim = kv.first, oldest = e.last_use;
        }
        if (!victim) return SIZE_MAX;
        drop_resident(victim);
    }
}

// A request that ends without a slot (refused at admission).
void Server::complete(const Request &r, mt_status st)
{
    mt_result res;
    std::memset(&res, 0, sizeof(res));
    res.status = st;
    res.root = 0xFFFFFFFFu;
    res.t_submit = r.t_submit;
    res.t_admit = res.t_done = now_s();
    done[r.ticket] = res;
    cv_done.notify_all();
}

Server::Admit Server::admit(Slot &s, const Request &r, mt_status &fail)
{
    const uint64_t n = (uint64_t)r.g.nx * r.g.ny * r.g.nz;
    mt_grid g = r.g;
    const size_t wsb = mt_workspace_bytes(g);
    const uint64_t cap = n / 2 + 1;  // minima are never adjacent: fewer than n/2 pairs
    Resident *res = nullptr;
    bool builds = true;
    if (r.key) {
        auto it = resident.find(r.key);
        if (it != resident.end()) {
            if (!same_grid(it->second.g, g)) {
                fail = MT_ERR_INVALID;  // a key names one field
                return kFailed;
            }
            if (!it->second.ready) return kWait;  // its building request is still running
            res = &it->second;
            builds = false;
        } else if (!r.h_f) {
            fail = MT_ERR_INVALID;  // not resident (any more) and no field given
            return kFailed;
        }
    }
    // this request's own buffers (labels, workspace), and for a build the
    // kept ones (field, triplets, pairs): one allocation for a one-off
    // request, two for a keyed build (the kept part outlives the request)
    const size_t own = own_bytes(n, wsb), kept = kept_bytes(n, cap);
    size_t off_own = SIZE_MAX, off_kept = SIZE_MAX;
    if (!r.key) {
        off_own = alloc_evicting(own + kept, 0);
        if (off_own == SIZE_MAX) return kNoRoom;
    } else {
        off_own = alloc_evicting(own, r.key);
        if (off_own == SIZE_MAX) return kNoRoom;
        if (builds) {
            off_kept = alloc_evicting(kept, r.key);
            if (off_kept == SIZE_MAX) {
                pool.release(off_own, own);
                return kNoRoom;
            }
        }
    }
    char *p = pool.base() + off_own;
    s.off = off_own;
    s.bytes = r.key ? own : own + kept;
    s.labels = reinterpret_cast<uint32_t *>(p);
    p += al256(4 * n);
    s.ws = p;
    p += al256(wsb);
    if (builds) {
        char *q = r.key ? pool.base() + off_kept : p;
        s.f = reinterpret_cast<float *>(q);
        q += al256(4 * n);
        s.W = reinterpret_cast<uint64_t *>(q);
        q += al256(8 * n);
        s.pairs = reinterpret_cast<uint32_t *>(q);
        if (r.key) {
            Resident &e = resident[r.key];
            e = Resident{};
            e.g = g;
            e.off = off_kept;
            e.bytes = kept;
            e.f = s.f, e.W = s.W, e.pairs = s.pairs;
            res = &e;
        }
    } else {
        s.f = res->f, s.W = res->W, s.pairs = res->pairs;
    }
    if (res) {
        res->users++;
        res->last_use = now_s();
    }
    s.builds = builds;
    s.ws_bytes = wsb;
    s.dev_cap = cap;
    s.req = r;
    s.t_admit = now_s();
    s.stage = 1;
    s.keep = MT_OK;
    std::memset(s.h_meta, 0, 4 * sizeof(uint64_t));
    cudaStream_t st = s.st;
    Workspace ws;
    bool ok = carve_workspace(s.ws, s.ws_bytes, n, ws);
    if (builds) {
        ok = ok && cudaMemcpyAsync(s.f, r.h_f, 4 * n, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && mt_build_triplets(s.f, g, s.W, s.ws, s.ws_bytes, st) == MT_OK;
        ok = ok && launch_pairs(s.W, n, s.pairs, cap, ws, st) == cudaSuccess;
    } else {
        s.h_meta[0] = res->npairs, s.h_meta[1] = res->nroots, s.h_meta[2] = res->root;
        ok = ok && cudaMemsetAsync(ws.status, 0, 256, st) == cudaSuccess;
    }
    ok = ok && mt_components_at(s.f, s.W, g, r.t, s.labels, s.ws, s.ws_bytes, st) == MT_OK;
    if (builds)
        ok = ok && cudaMemcpyAsync(s.h_meta, ws.meta, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(s.h_meta + 3, ws.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (r.h_labels)
        ok = ok && cudaMemcpyAsync(r.h_labels, s.labels, 4 * n, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaEventRecord(s.ev1, st) == cudaSuccess;
    if (!ok) {
        cudaStreamSynchronize(st);
        finish(s, MT_ERR_CUDA);
    }
    return kAdmitted;
}

void Server::finish(Slot &s, mt_status st)
{
    mt_result res;
    std::memset(&res, 0, sizeof(res));
    res.status = st;
    res.npairs = s.h_meta ? s.h_meta[0] : 0;
    res.root = (s.h_meta && s.h_meta[1] == 1) ? (uint32_t)s.h_meta[2] : 0xFFFFFFFFu;
    res.reused = s.builds ? 0u : 1u;
    res.t_submit = s.req.t_submit;
    res.t_admit = s.t_admit;
    res.t_done = now_s();
    pool.release(s.off, s.bytes);
    if (s.req.key) {
        auto it = resident.find(s.req.key);
        if (it != resident.end()) {
            Resident &e = it->second;
            e.users--;
            e.last_use = res.t_done;
            if (s.builds) {
                // the tree is kept only if it was built without error
                if (st == MT_OK || st == MT_ERR_CAPACITY) {
                    e.ready = true;
                    e.npairs = s.h_meta[0], e.nroots = s.h_meta[1], e.root = (uint32_t)s.h_meta[2];
                } else {
                    e.evict = true;
                }
            }
            if (e.evict && e.users == 0) drop_resident(s.req.key);
        }
    }
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
        // admit: arrival order, skipping requests that do not fit yet; a
        // request overtaken kMaxOvertakes times blocks admission behind it
        // until it fits
        for (auto it = pending.begin(); it != pending.end();) {
            Slot *free_slot = nullptr;
            for (auto &s : slots)
                if (s.stage == 0) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot) break;
            mt_status fail = MT_OK;
            const Admit a = admit(*free_slot, *it, fail);
            if (a == kAdmitted || a == kFailed) {
                if (a == kFailed) complete(*it, fail);
                // every request still waiting before this one was overtaken;
                // once one of them reaches the limit, nothing more is
                // admitted in this pass (the next pass starts with it)
                bool limit = false;
                for (auto jt = pending.begin(); jt != it; ++jt) limit |= ++jt->overtaken >= kMaxOvertakes;
                it = pending.erase(it);
                progressed = true;
                if (limit) break;
            } else if (a == kNoRoom && it->overtaken >= kMaxOvertakes) {
                break;
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

static mt_status submit(mt_server *srv, uint64_t key, const float *h_f, mt_grid g, float t, uint32_t *h_pairs,
                        uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket)
{
    if (!srv || (!h_f && !key) || !ticket || g.nx == 0 || g.ny == 0 || g.nz == 0 || t != t) return MT_ERR_INVALID;
    const uint64_t n = (uint64_t)g.nx * g.ny * g.nz;
    if (n >= 0xFFFFFFFFull) return MT_ERR_TOO_LARGE;
    Server &S = srv->s;
    if (request_bytes(n, mt_workspace_bytes(g), n / 2 + 1) > S.budget) return MT_ERR_NOMEM;
    std::lock_guard<std::mutex> lk(S.mu);
    Request r{S.next_ticket++, h_f, g, t, h_pairs, h_pairs ? pair_cap : 0, h_labels, now_s(), key, 0};
    S.pending.push_back(r);
    *ticket = r.ticket;
    S.cv_work.notify_one();
    return MT_OK;
}

mt_status mt_server_submit(mt_server *srv, const float *h_f, mt_grid g, float t, uint32_t *h_pairs,
                           uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket)
{
    return submit(srv, 0, h_f, g, t, h_pairs, pair_cap, h_labels, ticket);
}

mt_status mt_server_submit_resident(mt_server *srv, uint64_t key, const float *h_f, mt_grid g, float t,
                                    uint32_t *h_pairs, uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket)
{
    if (!key) return MT_ERR_INVALID;
    return submit(srv, key, h_f, g, t, h_pairs, pair_cap, h_labels, ticket);
}

mt_status mt_server_evict(mt_server *srv, uint64_t key)
{
    if (!srv || !key) return MT_ERR_INVALID;
    Server &S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.resident.find(key);
    if (it == S.resident.end()) return MT_ERR_INVALID;
    it->second.evict = true;
    if (it->second.users == 0) S.drop_resident(key);
    return MT_OK;
}

mt_status mt_server_resident(mt_server *srv, uint64_t *count, uint64_t *bytes)
{
    if (!srv || !count || !bytes) return MT_ERR_INVALID;
    Server &S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    uint64_t c = 0, b = 0;
    for (auto &kv : S.resident)
        if (kv.second.ready) c++, b += kv.second.bytes;
    *count = c;
    *bytes = b;
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
