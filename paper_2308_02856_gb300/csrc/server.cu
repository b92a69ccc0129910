// Serving: extraction jobs arrive over time and are hashed with continuous
// batching under a device-memory budget.
//
//  * submit() queues a job (the seed is copied; input and output stay in the
//    caller's device buffers).  A job that could never fit the budget is
//    refused with EXTRACT_EBUDGET.
//  * The scheduler thread admits queued jobs first-come first-served while
//    the budget (order + sub-block buffer + seed + the job's input and output)
//    and the slot count allow.
//  * A setup thread builds each admitted job's sampled order, copies its seed
//    and gathers its sub-blocks on its own stream, concurrently with hashing.
//  * Hashing runs in "waves": bounded launches of the persistent multi-job
//    kernel (batch.cu), each holding tiles of every ready job, shortest
//    remaining work first, up to a fixed amount of GPU time.  Jobs that become
//    ready join the next wave, so new work enters while older work is on the
//    GPU; two waves on two streams overlap so no SM idles between them.
//  * A job completes when the last wave holding its tiles has finished; its
//    memory goes back to the budget and waiters are woken.
// Results are bit-identical to extract_run: every tile of a job writes only
// that job's output, and partial parities combine by XOR in any order.
// No kernel waits on the host: each wave is an ordinary bounded launch.
#include "common.cuh"
#include "hash_tile.cuh"
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace ex {
namespace {

using Clock = std::chrono::steady_clock;

enum JobState { kQueued, kAdmitted, kSetupLaunched, kReady, kDone, kFailed };

constexpr int kWaveSlots = 2;
constexpr int kNttLanes = 2;
constexpr uint32_t kTcServeChunk = 32;  // K blocks of 128 per parity read-back of the tensor-core product
constexpr uint32_t kMaxWaveTiles = 1u << 16;

struct SJob {
    uint64_t ticket = 0;
    uint64_t n = 0, key = 0;
    uint32_t m = 0, s = 0, k = 0, flags = 0;
    const uint32_t *in = nullptr;
    uint32_t *out = nullptr;
    std::vector<uint32_t> seed_host;  // realigned seeds, nseeds x stride words
    uint32_t w_pad = 0, stride = 0, nseeds = 0, variant = 0;
    uint64_t bytes = 0;
    uint32_t *perm = nullptr, *arev = nullptr, *seed = nullptr;
    std::vector<BatchTileDev> tiles;  // job field filled per wave
    std::vector<double> tile_ns;      // GPU time of each tile
    size_t next_tile = 0;
    double remaining_ns = 0;
    int outstanding_waves = 0;
    JobState state = kQueued;
    int rc = EXTRACT_OK;
    cudaEvent_t setup_ev = nullptr;
    // NTT method or tensor-core product: hashed whole on a lane
    bool use_ntt = false, use_tc = false, hashed = false;
    bool on_lane() const { return use_ntt || use_tc; }
    NttPlan *ntt = nullptr;
    cudaEvent_t done_ev = nullptr;
    Clock::time_point t_submit, t_done;
};
using JobPtr = std::shared_ptr<SJob>;

struct NttLane {
    cudaStream_t st = nullptr;
    uint32_t *work = nullptr;
    JobPtr cur;
};

struct Wave {
    bool busy = false;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BatchJobDev *d_jobs = nullptr;
    BatchTileDev *d_tiles = nullptr;
    uint32_t *d_counter = nullptr;
    std::vector<JobPtr> jobs;
};

void realign_seed(const uint32_t *src, uint64_t src_words, uint64_t off, uint64_t len, uint32_t *dst,
                  uint64_t dst_words)
{
    std::memset(dst, 0, dst_words * 4);
    const uint64_t w0 = off >> 5;
    const uint32_t sh = (uint32_t)(off & 31u);
    const uint64_t nw = (len + 31) / 32;
    for (uint64_t t = 0; t < nw && t < dst_words; ++t) {
        const uint64_t a = w0 + t;
        const uint32_t lo = a < src_words ? src[a] : 0u, hi = a + 1 < src_words ? src[a + 1] : 0u;
        dst[t] = sh ? ((lo >> sh) | (hi << (32u - sh))) : lo;
    }
    if (len % 32 && nw - 1 < dst_words) dst[nw - 1] &= (1u << (len % 32)) - 1u;
}

// entries of a job's order: n (sorted order), m s (the i.i.d. law's padded
// order) or none (identity)
uint64_t order_entries(uint64_t n, uint32_t m, uint32_t s, uint32_t flags)
{
    if (flags & EXTRACT_IDENTITY_PERM) return 0;
    return (flags & EXTRACT_SAMPLING_IID) ? (uint64_t)m * s : n;
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace ex

using namespace ex;

struct extract_server {
    int device = 0, sms = 0;
    uint64_t budget = 0, in_use = 0, peak = 0;
    uint32_t max_slots = 0;
    double wave_ns = 0;        // GPU time per wave
    double tile_cap_sm_ns = 0; // SM time per tile
    const double *costs = nullptr;
    std::mutex mu;
    std::condition_variable cv_sched, cv_setup, cv_done;
    std::deque<JobPtr> pending, setup_q;
    std::vector<JobPtr> active;
    std::unordered_map<uint64_t, JobPtr> by_ticket;
    bool stop = false, setup_stop = false;
    uint64_t next_ticket = 1;
    cudaStream_t setup_st = nullptr;
    Wave waves[kWaveSlots];
    // lanes: one NTT or tensor-core job at a time each (own stream and NTT
    // work buffer), concurrent with the waves and with each other
    NttLane lanes[kNttLanes];
    uint32_t *d_err = nullptr;  // error word of the tensor-core kernels
    std::thread sched_thread, setup_thread;
    // statistics
    uint64_t submitted = 0, admitted = 0, completed = 0, failed = 0, rejected = 0, nwaves = 0;
    std::vector<double> latencies_ms;
    double bits_done = 0;
    bool any_submit = false;
    Clock::time_point first_submit, last_done;
};

namespace {

// Device work of one admitted job on the setup stream: seed, order, gather,
// cleared output.  Runs on the setup thread.
int setup_job(extract_server *S, SJob &J)
{
    cudaStream_t st = S->setup_st;
    EX_CUDA(cudaMallocAsync(&J.seed, J.seed_host.size() * 4, st));
    EX_CUDA(cudaMemcpyAsync(J.seed, J.seed_host.data(), J.seed_host.size() * 4, cudaMemcpyHostToDevice, st));
    EX_CUDA(cudaMallocAsync(&J.arev, (size_t)J.m * J.w_pad * 4, st));
    const bool iid = (J.flags & EXTRACT_SAMPLING_IID) != 0;
    if (!(J.flags & EXTRACT_IDENTITY_PERM)) {
        EX_CUDA(cudaMallocAsync(&J.perm, (size_t)order_entries(J.n, J.m, J.s, J.flags) * 4, st));
        const uint32_t kb = (J.flags >> 8) & 0x3fu;
        const uint64_t mask = kb ? ~((1ull << (64u - kb)) - 1ull) : ~0ull;
        if (iid) {
            std::vector<uint64_t> sizes;  // EXTRACT_EABORT fails the job
            if (int rc = build_iid_order(J.n, J.key, mask, J.m, J.s, J.perm, &sizes, st, S->sms)) return rc;
        } else if (int rc = build_perm(J.n, J.key, mask, J.perm, st, S->sms)) {
            return rc;
        }
    }
    if (int rc = launch_gather(J.in, J.perm, J.m, J.s, J.w_pad, J.arev, st, S->sms, 0, iid, J.n)) return rc;
    EX_CUDA(cudaMemsetAsync(J.out, 0, ceil_div((uint64_t)J.m * J.k, 32) * 4, st));
    if (J.use_ntt)  // tables and the seed spectrum (synchronous on the setup stream)
        if (int rc = ntt_create(&J.ntt, J.m, J.s, J.k, J.seed, st, S->lanes[0].work, -1, J.nseeds > 1 ? J.stride : 0))
            return rc;
    // the order is only needed by the gather: give its memory back now
    if (J.perm) {
        EX_CUDA(cudaFreeAsync(J.perm, st));
        J.perm = nullptr;
    }
    EX_CUDA(cudaEventRecord(J.setup_ev, st));
    return EXTRACT_OK;
}

void setup_loop(extract_server *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        JobPtr j;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_setup.wait(lk, [&] { return S->setup_stop || !S->setup_q.empty(); });
            if (S->setup_q.empty()) return;  // the scheduler has drained and stopped
            j = S->setup_q.front();
            S->setup_q.pop_front();
        }
        const int rc = setup_job(S, *j);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (rc != EXTRACT_OK) {
                j->rc = rc;
                j->state = kFailed;
            } else {
                j->state = kSetupLaunched;
            }
        }
        S->cv_sched.notify_all();
    }
}

// Frees go on the setup stream, after any setup work of the job; every wave
// that used the buffers has already completed.
void release_job(extract_server *S, SJob &J)
{
    cudaStream_t st = S->setup_st;
    if (J.perm) cudaFreeAsync(J.perm, st);
    if (J.arev) cudaFreeAsync(J.arev, st);
    if (J.seed) cudaFreeAsync(J.seed, st);
    J.perm = J.arev = J.seed = nullptr;
    if (J.ntt) {
        ntt_destroy_async(J.ntt, st);
        J.ntt = nullptr;
    }
    S->in_use -= J.bytes;
}

// Under S->mu.  Returns true if anything changed.
bool schedule_step(extract_server *S)
{
    bool progress = false;
    // 1. admission, first come first served
    while (!S->pending.empty() && S->active.size() < S->max_slots &&
           S->in_use + S->pending.front()->bytes <= S->budget) {
        JobPtr j = S->pending.front();
        S->pending.pop_front();
        S->in_use += j->bytes;
        S->peak = std::max(S->peak, S->in_use);
        j->state = kAdmitted;
        S->active.push_back(j);
        S->setup_q.push_back(j);
        ++S->admitted;
        S->cv_setup.notify_one();
        progress = true;
    }
    // 2. finished waves
    for (Wave &w : S->waves) {
        if (!w.busy) continue;
        const cudaError_t e = cudaEventQuery(w.ev);
        if (e == cudaErrorNotReady) continue;
        w.busy = false;
        progress = true;
        for (JobPtr &j : w.jobs) {
            --j->outstanding_waves;
            if (e != cudaSuccess && j->state != kFailed) {
                j->rc = cuda_error(e, "wave");
                j->state = kFailed;
            }
        }
        w.jobs.clear();
    }
    // 3. setups that finished; jobs that are complete or failed
    for (size_t i = 0; i < S->active.size();) {
        JobPtr j = S->active[i];
        if (j->state == kSetupLaunched) {
            const cudaError_t e = cudaEventQuery(j->setup_ev);
            if (e == cudaSuccess) {
                // the order was freed after the gather: return its share of the budget
                const uint64_t order_b = order_entries(j->n, j->m, j->s, j->flags) * 4;
                S->in_use -= order_b;
                j->bytes -= order_b;
                j->state = kReady;
                progress = true;
            }
            else if (e != cudaErrorNotReady) { j->rc = cuda_error(e, "setup"); j->state = kFailed; }
        }
        bool finished;
        if (j->on_lane()) {
            finished = false;
            if (j->state == kReady && j->hashed) {
                const cudaError_t e = cudaEventQuery(j->done_ev);
                if (e == cudaSuccess) {
                    finished = true;
                    uint32_t err = 0;  // a tensor-core kernel that gave up on a wait fails its job
                    uint32_t *ew = j->use_tc ? S->d_err : j->ntt ? ntt_error_word(j->ntt) : nullptr;
                    if (ew && cudaMemcpy(&err, ew, 4, cudaMemcpyDeviceToHost) == cudaSuccess && err) {
                        cudaMemset(ew, 0, 4);
                        j->rc = set_error(EXTRACT_ETIMEDOUT, "a tensor-core hash kernel gave up waiting");
                        j->state = kFailed;
                        finished = false;
                    }
                } else if (e != cudaErrorNotReady) {
                    j->rc = cuda_error(e, "lane job");
                    j->state = kFailed;
                }
            }
            if (finished || j->state == kFailed)
                for (NttLane &L : S->lanes)
                    if (L.cur == j) L.cur.reset();
        } else {
            finished = j->state == kReady && j->next_tile == j->tiles.size() && j->outstanding_waves == 0;
        }
        const bool dead = j->state == kFailed && j->outstanding_waves == 0;
        if (finished || dead) {
            release_job(S, *j);
            j->t_done = Clock::now();
            if (finished) {
                j->state = kDone;
                ++S->completed;
                S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count());
                S->bits_done += (double)j->n;
                S->last_done = j->t_done;
            } else {
                ++S->failed;
            }
            S->active.erase(S->active.begin() + (long)i);
            progress = true;
            S->cv_done.notify_all();
            continue;
        }
        ++i;
    }
    // 4. each free lane takes the ready lane job with the least predicted time
    for (NttLane &L : S->lanes) {
        if (L.cur) continue;
        JobPtr best;
        for (JobPtr &j : S->active)
            if (j->on_lane() && j->state == kReady && !j->hashed && (!best || j->remaining_ns < best->remaining_ns))
                best = j;
        if (!best) break;
        int rc = best->use_tc
                     ? launch_hash_tc(best->seed, best->stride, best->arev, best->w_pad, best->m, best->s, best->k,
                                      best->out, S->d_err, L.st, kTcServeChunk)
                     : ntt_hash(best->ntt, best->arev, best->w_pad, best->m, best->s, best->k, best->out, L.st, L.work);
        cudaError_t e = rc == EXTRACT_OK ? cudaEventRecord(best->done_ev, L.st) : cudaSuccess;
        if (rc == EXTRACT_OK && e != cudaSuccess) rc = cuda_error(e, "lane event");
        best->hashed = true;
        if (rc != EXTRACT_OK) {
            best->rc = rc;
            best->state = kFailed;
        } else {
            L.cur = best;
        }
        progress = true;
    }
    // 5. a new wave on a free slot: shortest remaining work first
    for (Wave &w : S->waves) {
        if (w.busy) continue;
        std::vector<JobPtr> ready;
        for (JobPtr &j : S->active)
            if (j->state == kReady && j->next_tile < j->tiles.size()) ready.push_back(j);
        if (ready.empty()) break;
        std::sort(ready.begin(), ready.end(),
                  [](const JobPtr &a, const JobPtr &b) { return a->remaining_ns < b->remaining_ns; });
        std::vector<BatchJobDev> table;
        std::vector<BatchTileDev> tiles;
        double used = 0;
        for (JobPtr &j : ready) {
            if (used >= S->wave_ns || tiles.size() >= kMaxWaveTiles || table.size() >= S->max_slots) break;
            const uint32_t jid = (uint32_t)table.size();
            BatchJobDev T{};
            T.seed = j->seed; T.arev = j->arev; T.out = j->out;
            T.seed_stride = j->nseeds > 1 ? j->stride : 0u;
            T.m = j->m; T.s = j->s; T.k = j->k; T.w_pad = j->w_pad;
            table.push_back(T);
            while (j->next_tile < j->tiles.size() && used < S->wave_ns && tiles.size() < kMaxWaveTiles) {
                BatchTileDev t = j->tiles[j->next_tile];
                t.job = jid;
                tiles.push_back(t);
                used += j->tile_ns[j->next_tile];
                j->remaining_ns -= j->tile_ns[j->next_tile];
                ++j->next_tile;
            }
            ++j->outstanding_waves;
            w.jobs.push_back(j);
        }
        // longest tiles first inside the wave
        std::vector<size_t> idx(tiles.size());
        for (size_t t = 0; t < idx.size(); ++t) idx[t] = t;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
            return (tiles[a].c_end - tiles[a].c_begin) > (tiles[b].c_end - tiles[b].c_begin);
        });
        std::vector<BatchTileDev> sorted(tiles.size());
        for (size_t t = 0; t < idx.size(); ++t) sorted[t] = tiles[idx[t]];
        cudaError_t e = cudaMemcpyAsync(w.d_jobs, table.data(), sizeof(BatchJobDev) * table.size(),
                                        cudaMemcpyHostToDevice, w.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w.d_tiles, sorted.data(), sizeof(BatchTileDev) * sorted.size(),
                                cudaMemcpyHostToDevice, w.st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.d_counter, 0, 4, w.st);
        int rc = e == cudaSuccess ? EXTRACT_OK : cuda_error(e, "wave upload");
        if (rc == EXTRACT_OK) rc = launch_batch_hash(w.d_jobs, w.d_tiles, (uint32_t)sorted.size(), w.d_counter,
                                                     S->sms, w.st);
        if (rc == EXTRACT_OK && (e = cudaEventRecord(w.ev, w.st)) != cudaSuccess) rc = cuda_error(e, "wave event");
        if (rc != EXTRACT_OK)
            for (JobPtr &j : w.jobs) { j->rc = rc; j->state = kFailed; --j->outstanding_waves; }
        else
            w.busy = true;
        if (rc != EXTRACT_OK) w.jobs.clear();
        ++S->nwaves;
        progress = true;
    }
    return progress;
}

void sched_loop(extract_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        const bool progress = schedule_step(S);
        if (S->stop && S->pending.empty() && S->active.empty()) break;
        if (!progress) {
            const bool idle = S->active.empty() && S->pending.empty();
            if (idle) S->cv_sched.wait(lk);
            else S->cv_sched.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

void destroy_server(extract_server *S)
{
    for (Wave &w : S->waves) {
        if (w.ev) cudaEventDestroy(w.ev);
        cudaFree(w.d_jobs);
        cudaFree(w.d_tiles);
        cudaFree(w.d_counter);
        if (w.st) cudaStreamDestroy(w.st);
    }
    if (S->setup_st) cudaStreamDestroy(S->setup_st);
    for (NttLane &L : S->lanes) {
        if (L.st) cudaStreamDestroy(L.st);
        cudaFree(L.work);
    }
    cudaFree(S->d_err);
    for (auto &kv : S->by_ticket) {
        if (kv.second->setup_ev) cudaEventDestroy(kv.second->setup_ev);
        if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    }
    delete S;
}

}  // namespace

extern "C" {

int extract_server_create(extract_server **out, uint64_t hbm_budget_bytes, uint32_t max_slots, uint32_t wave_us,
                          uint32_t flags)
{
    if (!out) return set_error(EXTRACT_EINVAL, "out is null");
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_slots == 0) return set_error(EXTRACT_EINVAL, "zero budget or slots");
    if (flags) return set_error(EXTRACT_EINVAL, "unknown server flags 0x%x", flags);
    extract_server *S = new (std::nothrow) extract_server();
    if (!S) return set_error(EXTRACT_ENOMEM, "host allocation failed");
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->wave_ns = (wave_us ? wave_us : 2000u) * 1e3;
    S->tile_cap_sm_ns = S->wave_ns / 8.0;  // SM time per tile: at least 8 tiles per SM per wave
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (e != cudaSuccess) { delete S; return cuda_error(e, "device query"); }
    if (int rc = tile_costs(S->device, S->sms, &S->costs)) { delete S; return rc; }
    int rc = EXTRACT_OK;
    do {
        if ((e = cudaStreamCreateWithFlags(&S->setup_st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_error(e, "stream"); break; }
        // each lane holds the largest NTT work buffer any job can need
        for (NttLane &L : S->lanes) {
            if ((e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_error(e, "stream"); break; }
            if ((e = cudaMalloc(&L.work, ntt_max_work_words() * 4)) != cudaSuccess) { rc = cuda_error(e, "ntt work"); break; }
        }
        if (rc != EXTRACT_OK) break;
        if ((e = cudaMalloc(&S->d_err, 4)) != cudaSuccess || (e = cudaMemset(S->d_err, 0, 4)) != cudaSuccess) {
            rc = cuda_error(e, "tensor-core error word");
            break;
        }
        for (Wave &w : S->waves) {
            if ((e = cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_error(e, "stream"); break; }
            if ((e = cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming)) != cudaSuccess) { rc = cuda_error(e, "event"); break; }
            if ((e = cudaMalloc(&w.d_jobs, sizeof(BatchJobDev) * max_slots)) != cudaSuccess) { rc = cuda_error(e, "wave jobs"); break; }
            if ((e = cudaMalloc(&w.d_tiles, sizeof(BatchTileDev) * kMaxWaveTiles)) != cudaSuccess) { rc = cuda_error(e, "wave tiles"); break; }
            if ((e = cudaMalloc(&w.d_counter, 4)) != cudaSuccess) { rc = cuda_error(e, "wave counter"); break; }
        }
    } while (0);
    if (rc != EXTRACT_OK) { destroy_server(S); return rc; }
    S->setup_thread = std::thread(setup_loop, S);
    S->sched_thread = std::thread(sched_loop, S);
    *out = S;
    return EXTRACT_OK;
}

int extract_server_submit(extract_server *S, const extract_job_desc *d, const uint32_t *in_bits_dev,
                          uint32_t *out_bits_dev, uint64_t *ticket)
{
    if (!S || !d || !ticket) return set_error(EXTRACT_EINVAL, "null argument");
    if (!in_bits_dev || !out_bits_dev || !d->seed_bits_host) return set_error(EXTRACT_EINVAL, "null buffer");
    const uint32_t known = EXTRACT_SEED_PER_SUBBLOCK | EXTRACT_IDENTITY_PERM | EXTRACT_SAMPLING_IID | (0x3fu << 8);
    if (d->flags & ~known) return set_error(EXTRACT_EINVAL, "unknown flags 0x%x", d->flags);
    const bool iid = (d->flags & EXTRACT_SAMPLING_IID) != 0;
    if (d->m < 1 || d->s < 1 || d->k < 1 || d->k > d->s || d->n > (1ull << 32) || (!iid && (uint64_t)d->m * d->s > d->n))
        return set_error(EXTRACT_EINVAL, "bad shape n=%llu m=%u s=%u k=%u", (unsigned long long)d->n, d->m, d->s, d->k);
    if (iid && ((d->flags & EXTRACT_IDENTITY_PERM) || d->n >= (1ull << 32) || d->m > (1u << 16)))
        return set_error(EXTRACT_EINVAL, "the i.i.d. law needs n < 2^32, m <= 2^16 and no identity order");
    JobPtr j = std::make_shared<SJob>();
    j->n = d->n; j->m = d->m; j->s = d->s; j->k = d->k; j->flags = d->flags; j->key = d->sampling_key;
    j->in = in_bits_dev;
    j->out = out_bits_dev;
    const bool per_sub = (d->flags & EXTRACT_SEED_PER_SUBBLOCK) != 0;
    j->w_pad = (uint32_t)round_up(ceil_div(d->s, 32), kWordChunk);
    j->variant = (uint32_t)choose_variant(d->m, d->k, j->w_pad, per_sub, S->costs);
    {
        const double tiles = (double)ceil_div(d->k, variant_rows((int)j->variant)) *
                             (double)ceil_div(d->m, (uint32_t)variant_j((int)j->variant));
        const double direct_ns = tiles * (j->w_pad / kWordChunk) * S->costs[j->variant];
        // the least predicted time of the three methods (the tensor-core
        // product only with a shared seed)
        const double ntt_ns = ntt_shape(d->s, d->k, -1, per_sub).N != 0
                                  ? predict_ntt_s(d->m, d->s, d->k, -1, per_sub) * 1e9 : 1e300;
        const double tc_ns = per_sub ? 1e300 : predict_tc_s(d->m, d->k, d->s) * 1e9;
        j->use_ntt = ntt_ns < direct_ns && ntt_ns <= tc_ns;
        j->use_tc = !j->use_ntt && tc_ns < direct_ns;
        if (j->use_ntt) j->remaining_ns = ntt_ns;
        if (j->use_tc) j->remaining_ns = tc_ns;
    }
    HashPlan vp;
    vp.q = variant_q(j->variant);
    vp.j = variant_j(j->variant);
    vp.gx = (uint32_t)ceil_div(d->k, vp.rows());
    j->stride = seed_stride_words(vp, d->k, j->w_pad);
    j->nseeds = per_sub ? d->m : 1u;
    const uint64_t L = (uint64_t)d->s + d->k - 1;
    try {
        j->seed_host.resize((size_t)j->nseeds * j->stride);
    } catch (...) {
        return set_error(EXTRACT_ENOMEM, "host allocation failed");
    }
    const uint64_t src_words = ceil_div(L * j->nseeds, 32);
    for (uint32_t q = 0; q < j->nseeds; ++q)
        realign_seed(d->seed_bits_host, src_words, (uint64_t)q * L, L, j->seed_host.data() + (size_t)q * j->stride,
                     j->stride);
    // budget charge: order (freed early, still charged) + sub-blocks + seed + the job's input and output
    const uint64_t order_b = order_entries(d->n, d->m, d->s, d->flags) * 4;
    j->bytes = order_b + (uint64_t)d->m * j->w_pad * 4 + (uint64_t)j->seed_host.size() * 4 + ceil_div(d->n, 32) * 4 +
               ceil_div((uint64_t)d->m * d->k, 32) * 4 + (j->use_ntt ? ntt_plan_bytes(d->s, d->k, -1, per_sub) : 0);
    // tiles: every (row tile, sub-block tile, word range), each about tile_cap of one SM
    const uint32_t rows = vp.rows(), J = (uint32_t)vp.j, nchunks = j->w_pad / kWordChunk;
    const double ns_chunk = S->costs[j->variant];  // GPU ns per CTA-chunk
    const uint32_t cps = (uint32_t)std::max<double>(1.0, std::min<double>(nchunks,
                                                        S->tile_cap_sm_ns / (ns_chunk * S->sms)));
    const uint32_t gx = (uint32_t)ceil_div(d->k, rows), gy = (uint32_t)ceil_div(d->m, J);
    for (uint32_t by = 0; by < gy && !j->on_lane(); ++by)
        for (uint32_t bx = 0; bx < gx; ++bx)
            for (uint32_t c = 0; c < nchunks; c += cps) {
                const uint32_t ce = std::min(nchunks, c + cps);
                j->tiles.push_back(BatchTileDev{0u, j->variant, bx * rows, by * J, c, ce});
                j->tile_ns.push_back((ce - c) * ns_chunk);
                j->remaining_ns += (ce - c) * ns_chunk;
            }
    cudaError_t e = cudaEventCreateWithFlags(&j->setup_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (j->setup_ev) cudaEventDestroy(j->setup_ev);
        return cuda_error(e, "event");
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        cudaEventDestroy(j->setup_ev);
        cudaEventDestroy(j->done_ev);
        return set_error(EXTRACT_EBUSY, "server is stopping");
    }
    if (j->bytes > S->budget) {
        ++S->rejected;
        cudaEventDestroy(j->setup_ev);
        cudaEventDestroy(j->done_ev);
        return set_error(EXTRACT_EBUDGET, "job needs %llu bytes, budget is %llu", (unsigned long long)j->bytes,
                         (unsigned long long)S->budget);
    }
    j->ticket = S->next_ticket++;
    j->t_submit = Clock::now();
    if (!S->any_submit) { S->any_submit = true; S->first_submit = j->t_submit; }
    ++S->submitted;
    S->pending.push_back(j);
    S->by_ticket[j->ticket] = j;
    *ticket = j->ticket;
    S->cv_sched.notify_all();
    return EXTRACT_OK;
}

int extract_server_wait(extract_server *S, uint64_t ticket, uint32_t timeout_ms, double *latency_ms)
{
    if (!S) return set_error(EXTRACT_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return set_error(EXTRACT_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    JobPtr j = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return j->state == kDone || (j->state == kFailed && j->outstanding_waves == 0 && j->t_done != Clock::time_point()); });
    if (!ok) return set_error(EXTRACT_ETIMEDOUT, "ticket %llu not done after %u ms", (unsigned long long)ticket,
                              timeout_ms);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    const int rc = j->rc;
    if (j->setup_ev) { cudaEventDestroy(j->setup_ev); j->setup_ev = nullptr; }
    if (j->done_ev) { cudaEventDestroy(j->done_ev); j->done_ev = nullptr; }
    S->by_ticket.erase(it);
    if (j->state == kFailed) return set_error(rc ? rc : EXTRACT_EINTERNAL, "ticket %llu failed",
                                              (unsigned long long)ticket);
    return EXTRACT_OK;
}

int extract_server_stats(extract_server *S, extract_stats *st)
{
    if (!S || !st) return set_error(EXTRACT_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->admitted = S->admitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->rejected = S->rejected;
    st->queued = S->pending.size();
    st->active = S->active.size();
    st->waves = S->nwaves;
    st->bytes_in_use = S->in_use;
    st->bytes_peak = S->peak;
    st->p50_ms = percentile(S->latencies_ms, 0.50);
    st->p99_ms = percentile(S->latencies_ms, 0.99);
    double sum = 0, mx = 0;
    for (double v : S->latencies_ms) { sum += v; mx = std::max(mx, v); }
    st->mean_ms = S->latencies_ms.empty() ? 0 : sum / (double)S->latencies_ms.size();
    st->max_ms = mx;
    st->input_bits_done = S->bits_done;
    if (S->completed && S->any_submit) {
        st->span_s = std::chrono::duration<double>(S->last_done - S->first_submit).count();
        st->gbit_per_s = st->span_s > 0 ? S->bits_done / st->span_s / 1e9 : 0;
    }
    return EXTRACT_OK;
}

int extract_server_destroy(extract_server *S)
{
    if (!S) return EXTRACT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    S->cv_setup.notify_all();
    if (S->sched_thread.joinable()) S->sched_thread.join();  // drains every submitted job
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->setup_stop = true;
    }
    S->cv_setup.notify_all();
    if (S->setup_thread.joinable()) S->setup_thread.join();
    const cudaError_t e = cudaDeviceSynchronize();
    destroy_server(S);
    if (e != cudaSuccess) return cuda_error(e, "server destroy");
    return EXTRACT_OK;
}

}  // extern "C"
