// serve.cu -- search-request serving with continuous batching.
//
// A request is one test-time search (App. E): a root position, K belief
// samples and a rollout depth; its result is the win/loss/draw/unfinished
// tally of st_rollout for the same inputs.
//
// Device-resident state: a table of request slots (root position, root state
// built on the GPU, per-request counters) and a pool of per-sample records
// (the sampled hidden types and the outcome of each rollout), both allocated
// once at create time.  A request is admitted when a request slot, K
// contiguous sample records and a launch slot are free, so admission is by
// free device memory.
//
// A host scheduler thread admits every request that fits, in arrival order,
// and issues one batch (root kernel + rollout kernel, one 8-lane team per
// (request, sample) at a time on at most a resident grid) for all requests
// admitted since the previous batch, on the next stream of a pool.
// Submissions wait under their own small lock, so a submit never waits for
// a scheduler pass.  Batches already running keep running: new requests
// never wait for a batch boundary, their work overlaps the older work on the
// GPU, and the slots of a finished request are reused at once.  The team that
// finishes a request's last rollout copies the tallies to host-mapped memory
// and then publishes a completion word; the scheduler polls those words.  No
// kernel ever waits on the host or on another kernel.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include "rollout.cuh"
#include "host_common.h"

using namespace stg;

namespace {

struct __align__(16) ReqDesc {
    int32_t K;
    int32_t depth;
    uint32_t k0, k1;
    uint32_t stream;
    uint32_t seq;          // completion word value for this admission
    int32_t sample_base;   // first sample record
    int32_t remaining;     // rollouts still running
    int32_t tallies[4];
};

struct __align__(16) SampleRec {
    uint8_t types[40];
    int8_t outcome;
    uint8_t pad[7];
};

struct __align__(16) BatchEntry {
    int32_t slot;
    int32_t unit_begin;    // prefix sum of K over the batch
};

struct __align__(16) Staged {
    st_position pos;
    ReqDesc desc;
};

__global__ void k_serve_roots(const BatchEntry* entries, int n, const Staged* staged, RootState* roots,
                              ReqDesc* descs, volatile int32_t* host_tallies, volatile uint32_t* host_done)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int slot = entries[i].slot;
    build_root(S, &staged[slot].pos, roots + slot);
    if (lane_id() == 0) {
        descs[slot] = staged[slot].desc;
        if (staged[slot].desc.K == 0) {
            // no rollout will run: publish an empty result here (bad positions are marked by -1)
            const int32_t mark = roots[slot].bad ? -1 : 0;
            for (int j = 0; j < 4; ++j) host_tallies[4 * slot + j] = mark;
            __threadfence_system();
            host_done[slot] = staged[slot].desc.seq;
        }
    }
}

constexpr int kServeLanes = 8;   // one rollout per 8-lane team
constexpr int kServeWarps = 2;
constexpr int kServeTeams = 32 * kServeWarps / kServeLanes;   // rollouts per block
constexpr int kServeMinBlocks = 12;                           // resident blocks per SM the registers allow

// One (request, sample) unit per 8-lane team at a time, striding over the
// batch's units with at most a resident grid; the team's chase store is its
// slot of this launch slot's scratch (the newest four entries stay cached
// in shared memory).
__global__ void __launch_bounds__(32 * kServeWarps, kServeMinBlocks)
k_serve_rollouts(const BatchEntry* entries, int n, long long units, const RootState* roots, ReqDesc* descs,
                 SampleRec* samples, Rules Rl, volatile int32_t* host_tallies, volatile uint32_t* host_done,
                 uint64_t* pi_scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<kServeLanes> T;
    const int team = threadIdx.x / kServeLanes;
    FlatSmem* S = reinterpret_cast<FlatSmem*>(smem) + team;
    uint64_t* pi = pi_scratch + ((size_t)blockIdx.x * kServeTeams + team) * kPiWords;
    const int lane = T.tl;
    const long long stride = (long long)gridDim.x * kServeTeams;
    for (long long u = (long long)blockIdx.x * kServeTeams + team; u < units; u += stride) {
        // the batch entry holding unit u
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (entries[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
        }
        const int slot = entries[lo].slot;
        const RootState* R = roots + slot;
        ReqDesc* d = descs + slot;
        const int k = (int)(u - entries[lo].unit_begin);
        const bool bad = R->bad != 0;
        if (!bad) {
            const int outcome = rollout_one(&S->g, S->types, pi, (uint16_t*)nullptr, T, R, &R->plan, nullptr,
                                            d->depth, d->k0, d->k1, d->stream, (uint32_t)k, Rl);
            SampleRec* rec = samples + d->sample_base + k;
            for (int i = lane; i < 10; i += kServeLanes)
                reinterpret_cast<uint32_t*>(rec->types)[i] = reinterpret_cast<const uint32_t*>(S->types)[i];
            if (lane == 0) {
                rec->outcome = (int8_t)outcome;
                atomicAdd(&d->tallies[outcome], 1);
            }
        }
        // every unit of the request counts down, so the slot is reused only
        // after all of its units are done; the last one publishes the result
        if (lane == 0) {
            __threadfence();
            if (atomicSub(&d->remaining, 1) == 1) {
                __threadfence();
                for (int j = 0; j < 4; ++j) host_tallies[4 * slot + j] = bad ? -1 : atomicAdd(&d->tallies[j], 0);
                __threadfence_system();
                host_done[slot] = d->seq;
            }
        }
        T.sync();
    }
}

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
    st_request req;
    uint64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
    int slot = -1;
    int sample_base = 0;
    uint32_t seq = 0;
    int state = 0;            // 0 queued, 1 running, 2 done, 3 failed
    st_status status = ST_OK;
    int32_t tallies[4] = {0, 0, 0, 0};
};

}  // namespace

struct st_server {
    st_serve_config cfg{};
    Rules rules{};
    // device
    RootState* roots = nullptr;
    ReqDesc* descs = nullptr;
    SampleRec* samples = nullptr;
    Staged* staged_dev = nullptr;
    BatchEntry* entries_dev = nullptr;       // [max_batches][max_requests]
    // host pinned
    Staged* staged_host = nullptr;
    BatchEntry* entries_host = nullptr;      // [max_batches][max_requests]
    int32_t* host_tallies = nullptr;         // mapped [max_requests][4]
    uint32_t* host_done = nullptr;           // mapped [max_requests]
    int32_t* host_tallies_dev = nullptr;
    uint32_t* host_done_dev = nullptr;
    uint64_t* pi_scratch = nullptr;          // [max_batches][max_grid * kServeTeams][kPiWords]
    int max_grid = 0;                        // resident blocks of the rollout kernel
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> batch_done;
    std::vector<int> stream_busy;
    // host bookkeeping (guarded by mu)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<uint64_t> slot_ticket;       // ticket running in each request slot (0 free)
    std::map<int, int> free_ranges;          // sample records: begin -> length
    uint32_t next_seq = 1;
    bool stop = false;
    std::atomic<bool> failed{false};
    // submissions land here under their own lock, so a submit never waits
    // for a scheduler pass; the scheduler moves them into `tickets`/`queue`
    std::mutex in_mu;
    std::deque<std::pair<uint64_t, Ticket>> incoming;
    std::atomic<uint64_t> next_ticket{1};
    std::atomic<int64_t> n_incoming{0};
    std::atomic<bool> idle{false};           // the scheduler is (about to be) blocked on cv
    std::string fail_msg;
    st_serve_stats stats{};
    std::thread worker;
    int next_stream = 0;
};

namespace {

int take_range(st_server* s, int k)
{
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second >= k) {
            const int b = it->first, len = it->second;
            s->free_ranges.erase(it);
            if (len > k) s->free_ranges[b + k] = len - k;
            return b;
        }
    }
    return -1;
}

void give_range(st_server* s, int b, int k)
{
    if (k <= 0) return;
    auto it = s->free_ranges.emplace(b, k).first;
    auto nx = std::next(it);
    if (nx != s->free_ranges.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_ranges.erase(nx);
    }
    if (it != s->free_ranges.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_ranges.erase(it);
        }
    }
}

// One pass of the scheduler: retire finished requests and batches, admit and
// launch.  Returns whether anything is still in flight.  Called with mu held.
bool schedule_once(st_server* s, std::unique_lock<std::mutex>& lk)
{
    const int R = s->cfg.max_requests;
    // take in the new submissions, in submission order
    if (s->n_incoming.load() > 0) {
        std::lock_guard<std::mutex> g(s->in_mu);
        for (auto& kv : s->incoming) {
            s->tickets.emplace(kv.first, kv.second);
            s->queue.push_back(kv.first);
            s->stats.submitted += 1;
        }
        s->n_incoming.fetch_sub((int64_t)s->incoming.size());
        s->incoming.clear();
    }
    // retire requests whose completion word arrived
    for (int slot = 0; slot < R; ++slot) {
        const uint64_t t = s->slot_ticket[slot];
        if (!t) continue;
        Ticket& tk = s->tickets[t];
        const uint32_t seen = reinterpret_cast<volatile uint32_t*>(s->host_done)[slot];
        if (seen != tk.seq) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        for (int j = 0; j < 4; ++j) tk.tallies[j] = reinterpret_cast<volatile int32_t*>(s->host_tallies)[4 * slot + j];
        tk.done_ns = now_ns();
        if (tk.tallies[0] < 0) { tk.state = 3; tk.status = ST_ERR_BAD_POSITION; for (int j = 0; j < 4; ++j) tk.tallies[j] = 0; }
        else tk.state = 2;
        s->stats.completed += 1;
        give_range(s, tk.sample_base, tk.req.K);
        s->slot_ticket[slot] = 0;
        s->cv.notify_all();
    }
    // recycle launch slots whose batch finished
    bool inflight = false;
    for (size_t b = 0; b < s->streams.size(); ++b) {
        if (!s->stream_busy[b]) continue;
        const cudaError_t q = cudaEventQuery(s->batch_done[b]);
        if (q == cudaSuccess) s->stream_busy[b] = 0;
        else if (q == cudaErrorNotReady) inflight = true;
        else { s->failed = true; s->fail_msg = cudaGetErrorString(q); s->stream_busy[b] = 0; }
    }
    for (int slot = 0; slot < R; ++slot) inflight |= s->slot_ticket[slot] != 0;
    if (s->queue.empty()) return inflight;
    // a free launch slot
    int b = -1;
    for (size_t i = 0; i < s->streams.size(); ++i) {
        const int c = (s->next_stream + (int)i) % (int)s->streams.size();
        if (!s->stream_busy[c]) { b = c; break; }
    }
    if (b < 0) return true;
    // admit in arrival order while slots and sample records are free
    BatchEntry* ent = s->entries_host + (size_t)b * R;
    int n = 0;
    long long units = 0;
    while (!s->queue.empty() && n < R) {
        const uint64_t t = s->queue.front();
        Ticket& tk = s->tickets[t];
        int slot = -1;
        for (int i = 0; i < R; ++i)
            if (!s->slot_ticket[i]) { slot = i; break; }
        if (slot < 0) break;
        const int base = tk.req.K > 0 ? take_range(s, tk.req.K) : 0;
        if (base < 0) break;
        s->queue.pop_front();
        tk.slot = slot;
        tk.sample_base = base;
        tk.seq = s->next_seq++;
        if (s->next_seq == 0) s->next_seq = 1;
        tk.state = 1;
        tk.admit_ns = now_ns();
        s->slot_ticket[slot] = t;
        Staged& st = s->staged_host[slot];
        st.pos = tk.req.pos;
        std::memset(&st.desc, 0, sizeof(st.desc));
        st.desc.K = tk.req.K;
        st.desc.depth = tk.req.depth;
        st.desc.k0 = (uint32_t)tk.req.seed;
        st.desc.k1 = (uint32_t)(tk.req.seed >> 32);
        st.desc.stream = tk.req.stream_id;
        st.desc.seq = tk.seq;
        st.desc.sample_base = base;
        st.desc.remaining = tk.req.K;
        ent[n].slot = slot;
        ent[n].unit_begin = (int32_t)units;
        units += tk.req.K;
        ++n;
        s->stats.admitted += 1;
    }
    if (n == 0) return true;
    s->stats.batches += 1;
    s->stats.max_batch_requests = std::max<int64_t>(s->stats.max_batch_requests, n);
    cudaStream_t str = s->streams[b];
    // enqueue without the lock: copies, roots, rollouts, completion event
    lk.unlock();
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        const int slot = ent[i].slot;
        err = cudaMemcpyAsync(s->staged_dev + slot, s->staged_host + slot, sizeof(Staged), cudaMemcpyHostToDevice, str);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(s->entries_dev + (size_t)b * R, ent, n * sizeof(BatchEntry), cudaMemcpyHostToDevice, str);
    if (err == cudaSuccess) {
        const int rb = (n + 3) / 4;
        k_serve_roots<<<rb, 128, 4 * sizeof(RolloutSmem), str>>>(s->entries_dev + (size_t)b * R, n, s->staged_dev,
                                                                 s->roots, s->descs, s->host_tallies_dev,
                                                                 s->host_done_dev);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess && units > 0) {
        const long long fb = std::min((units + kServeTeams - 1) / kServeTeams, (long long)s->max_grid);
        k_serve_rollouts<<<(unsigned)fb, 32 * kServeWarps, kServeTeams * sizeof(FlatSmem), str>>>(
            s->entries_dev + (size_t)b * R, n, units, s->roots, s->descs, s->samples, s->rules, s->host_tallies_dev,
            s->host_done_dev, s->pi_scratch + (size_t)b * s->max_grid * kServeTeams * kPiWords);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(s->batch_done[b], str);
    lk.lock();
    if (err != cudaSuccess) {
        s->failed = true;
        s->fail_msg = cudaGetErrorString(err);
    }
    s->stream_busy[b] = 1;
    s->next_stream = (b + 1) % (int)s->streams.size();
    return true;
}

void worker_main(st_server* s)
{
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        const bool busy = schedule_once(s, lk);
        if (s->failed) {
            // fail every waiting and running request; nothing more is launched
            {
                std::lock_guard<std::mutex> g(s->in_mu);
                for (auto& kv : s->incoming) s->tickets.emplace(kv.first, kv.second);
                s->n_incoming.fetch_sub((int64_t)s->incoming.size());
                s->incoming.clear();
            }
            for (auto& kv : s->tickets)
                if (kv.second.state < 2) { kv.second.state = 3; kv.second.status = ST_ERR_CUDA; }
            s->queue.clear();
            s->cv.notify_all();
            s->cv.wait(lk, [s] { return s->stop; });
            break;
        }
        if (busy) {
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            s->idle.store(true);
            s->cv.wait_for(lk, std::chrono::milliseconds(5),
                           [s] { return s->stop || !s->queue.empty() || s->n_incoming.load() > 0; });
            s->idle.store(false);
        }
    }
}

}  // namespace

extern "C" st_status st_serve_create(const st_serve_config* cfg, st_server** out)
{
    ST_NVTX("st_serve_create");
    ST_CHECK_ARG(cfg && out, "st_serve_create: null argument");
    ST_CHECK_ARG(cfg->max_requests >= 1 && cfg->max_requests <= 65536, "st_serve_create: max_requests 1..65536");
    ST_CHECK_ARG(cfg->sample_slots >= 1 && cfg->sample_slots <= (1 << 26), "st_serve_create: sample_slots 1..2^26");
    ST_CHECK_ARG(cfg->max_batches >= 1 && cfg->max_batches <= 64, "st_serve_create: max_batches 1..64");
    ST_CHECK_ARG(rules_ok(&cfg->rules, true), "st_serve_create: invalid rules");
    int ndev = 0;
    ST_CUDA(cudaGetDeviceCount(&ndev));
    ST_CHECK_ARG(cfg->device >= 0 && cfg->device < ndev, "st_serve_create: device %d not present", cfg->device);
    *out = nullptr;
    ST_CUDA(cudaSetDevice(cfg->device));
    st_server* s = new st_server();
    s->cfg = *cfg;
    s->rules.k = cfg->rules.battleless_limit;
    s->rules.cap = cfg->rules.max_plies;
    s->rules.flags = cfg->rules.flags;
    const int R = cfg->max_requests, B = cfg->max_batches;
    cudaError_t err = cudaMalloc(&s->roots, (size_t)R * sizeof(RootState));
    if (err == cudaSuccess) err = cudaMalloc(&s->descs, (size_t)R * sizeof(ReqDesc));
    if (err == cudaSuccess) err = cudaMalloc(&s->samples, (size_t)cfg->sample_slots * sizeof(SampleRec));
    if (err == cudaSuccess) err = cudaMalloc(&s->staged_dev, (size_t)R * sizeof(Staged));
    if (err == cudaSuccess) err = cudaMalloc(&s->entries_dev, (size_t)B * R * sizeof(BatchEntry));
    if (err == cudaSuccess) {
        int occ = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve_rollouts, 32 * kServeWarps,
                                                            kServeTeams * sizeof(FlatSmem));
        s->max_grid = std::max(1, occ) * sm_count();
    }
    if (err == cudaSuccess)
        err = cudaMalloc(&s->pi_scratch, (size_t)B * s->max_grid * kServeTeams * kPiWords * sizeof(uint64_t));
    if (err == cudaSuccess) err = cudaHostAlloc(&s->staged_host, (size_t)R * sizeof(Staged), cudaHostAllocDefault);
    if (err == cudaSuccess) err = cudaHostAlloc(&s->entries_host, (size_t)B * R * sizeof(BatchEntry), cudaHostAllocDefault);
    if (err == cudaSuccess)
        err = cudaHostAlloc(&s->host_tallies, (size_t)R * 4 * sizeof(int32_t), cudaHostAllocMapped);
    if (err == cudaSuccess) err = cudaHostAlloc(&s->host_done, (size_t)R * sizeof(uint32_t), cudaHostAllocMapped);
    if (err == cudaSuccess) err = cudaHostGetDevicePointer(&s->host_tallies_dev, s->host_tallies, 0);
    if (err == cudaSuccess) err = cudaHostGetDevicePointer(&s->host_done_dev, s->host_done, 0);
    for (int b = 0; b < B && err == cudaSuccess; ++b) {
        cudaStream_t str;
        cudaEvent_t ev;
        err = cudaStreamCreateWithFlags(&str, cudaStreamNonBlocking);
        if (err != cudaSuccess) break;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err != cudaSuccess) {
            cudaStreamDestroy(str);   // not yet in the server's lists, which destroy frees
            break;
        }
        s->streams.push_back(str);
        s->batch_done.push_back(ev);
        s->stream_busy.push_back(0);
    }
    if (err != cudaSuccess) {
        stg::set_error("st_serve_create: %s", cudaGetErrorString(err));
        cudaGetLastError();
        st_serve_destroy(s);
        return ST_ERR_OOM;
    }
    std::memset(s->host_done, 0, (size_t)R * sizeof(uint32_t));
    std::memset(s->host_tallies, 0, (size_t)R * 4 * sizeof(int32_t));
    s->slot_ticket.assign(R, 0);
    s->free_ranges[0] = cfg->sample_slots;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return ST_OK;
}

extern "C" st_status st_serve_submit(st_server* s, const st_request* req, uint64_t* ticket)
{
    ST_NVTX("st_serve_submit");
    ST_CHECK_ARG(s && req && ticket, "st_serve_submit: null argument");
    ST_CHECK_ARG(req->K >= 0 && req->K <= s->cfg.sample_slots, "st_serve_submit: K %d outside 0..%d", req->K,
                 s->cfg.sample_slots);
    ST_CHECK_ARG(req->depth >= 0, "st_serve_submit: negative depth");
    if (s->failed.load()) {
        std::lock_guard<std::mutex> lk(s->mu);
        stg::set_error("st_serve_submit: server failed: %s", s->fail_msg.c_str());
        return ST_ERR_CUDA;
    }
    Ticket tk;
    tk.req = *req;
    tk.submit_ns = now_ns();
    uint64_t t = 0;
    {
        std::lock_guard<std::mutex> g(s->in_mu);
        if (s->incoming.size() >= 1u << 20) {
            stg::set_error("st_serve_submit: queue full");
            return ST_ERR_BUSY;
        }
        t = s->next_ticket.fetch_add(1);
        s->incoming.emplace_back(t, tk);
        s->n_incoming.fetch_add(1);
    }
    *ticket = t;
    // wake the scheduler only if it sleeps; taking mu once orders this
    // submission before its next look at n_incoming
    if (s->idle.load()) {
        { std::lock_guard<std::mutex> lk(s->mu); }
        s->cv.notify_all();
    }
    return ST_OK;
}

// Is the ticket submitted but not yet taken in by the scheduler?
static bool in_incoming(st_server* s, uint64_t ticket)
{
    std::lock_guard<std::mutex> g(s->in_mu);
    for (const auto& kv : s->incoming)
        if (kv.first == ticket) return true;
    return false;
}

static st_status take_result(st_server* s, uint64_t ticket, int32_t* tallies, st_timing* timing)
{
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        if (in_incoming(s, ticket)) return ST_ERR_NOT_READY;
        stg::set_error("st_serve: unknown ticket %llu", (unsigned long long)ticket);
        return ST_ERR_INVALID;
    }
    Ticket& tk = it->second;
    if (tk.state < 2) return ST_ERR_NOT_READY;
    if (tallies) std::memcpy(tallies, tk.tallies, sizeof(tk.tallies));
    if (timing) {
        timing->submit_ns = tk.submit_ns;
        timing->admit_ns = tk.admit_ns;
        timing->done_ns = tk.done_ns;
    }
    const st_status st = tk.state == 2 ? ST_OK : tk.status;
    if (st != ST_OK) stg::set_error("st_serve: request %llu failed", (unsigned long long)ticket);
    s->tickets.erase(it);
    return st;
}

extern "C" st_status st_serve_poll(st_server* s, uint64_t ticket, int32_t* tallies, st_timing* timing)
{
    ST_NVTX("st_serve_poll");
    ST_CHECK_ARG(s, "st_serve_poll: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    return take_result(s, ticket, tallies, timing);
}

extern "C" st_status st_serve_wait(st_server* s, uint64_t ticket, int32_t timeout_ms, int32_t* tallies,
                                   st_timing* timing)
{
    ST_NVTX("st_serve_wait");
    ST_CHECK_ARG(s, "st_serve_wait: null server");
    ST_CHECK_ARG(timeout_ms >= 0, "st_serve_wait: negative timeout");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end() && !in_incoming(s, ticket)) {
            stg::set_error("st_serve_wait: unknown ticket %llu", (unsigned long long)ticket);
            return ST_ERR_INVALID;
        }
        if (it != s->tickets.end() && it->second.state >= 2) return take_result(s, ticket, tallies, timing);
        if (it == s->tickets.end() && s->failed.load()) {
            stg::set_error("st_serve_wait: server failed: %s", s->fail_msg.c_str());
            return ST_ERR_CUDA;
        }
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = s->tickets.find(ticket);
            if (jt != s->tickets.end() && jt->second.state >= 2) return take_result(s, ticket, tallies, timing);
            stg::set_error("st_serve_wait: ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
            return ST_ERR_TIMEOUT;
        }
    }
}

extern "C" st_status st_serve_get_stats(st_server* s, st_serve_stats* out)
{
    ST_NVTX("st_serve_get_stats");
    ST_CHECK_ARG(s && out, "st_serve_get_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int64_t)s->queue.size() + s->n_incoming.load();
    int64_t running = 0;
    for (uint64_t t : s->slot_ticket) running += t != 0;
    out->running = running;
    return ST_OK;
}

extern "C" st_status st_serve_destroy(st_server* s)
{
    ST_NVTX("st_serve_destroy");
    if (!s) return ST_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->cfg.device);
    for (size_t b = 0; b < s->streams.size(); ++b) {
        cudaStreamSynchronize(s->streams[b]);
        cudaStreamDestroy(s->streams[b]);
        cudaEventDestroy(s->batch_done[b]);
    }
    cudaFree(s->roots); cudaFree(s->descs); cudaFree(s->samples); cudaFree(s->staged_dev); cudaFree(s->entries_dev);
    cudaFree(s->pi_scratch);
    cudaFreeHost(s->staged_host); cudaFreeHost(s->entries_host);
    cudaFreeHost(s->host_tallies); cudaFreeHost(s->host_done);
    delete s;
    return ST_OK;
}
