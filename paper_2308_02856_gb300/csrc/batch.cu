// Batching: many independent blocks of uneven n, s and k hashed in one
// persistent launch (Sec. III.B applied to many blocks at once).
//
// Per run, three kernels (captured once into a CUDA graph and replayed):
//   1. batch_zero_kernel   - clears every job's output and the tile counter;
//   2. batch_gather_kernel - gathers every job's sub-blocks (grid-stride over
//                            all jobs' 32-word groups);
//   3. batch_hash_kernel   - one CTA per SM pulls tiles from a global list
//                            (longest first) with an atomic counter; each
//                            tile runs the tile body of its job's variant.
// The per-run input/output pointers live in a device job table that is
// refreshed by one copy before the graph launch, so the graph never changes.
//
// Tile choice (the autotuner): every variant's cost per (CTA, word chunk) is
// measured once per device inside the persistent kernel itself; each job then
// takes the variant with the least predicted time (tiles x chunks x cost,
// padding included) and a word-range split that keeps every tile under a
// share of the batch so the longest-first order balances the SMs.
#include "common.cuh"
#include "gather_body.cuh"
#include "hash_tile.cuh"
#include "internal.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace ex {

namespace {

__device__ __forceinline__ uint32_t find_job(const BatchJobDev *jobs, uint32_t njobs, uint64_t x, bool by_groups)
{
    uint32_t lo = 0, hi = njobs - 1;  // last job whose prefix <= x
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        const uint64_t v = by_groups ? jobs[mid].groups_before : jobs[mid].outw_before;
        if (v <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_zero_kernel(const BatchJobDev *__restrict__ jobs, uint32_t njobs, uint64_t total_words,
                                  uint32_t *counter)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total_words; t += stride) {
        const uint32_t j = find_job(jobs, njobs, t, false);
        jobs[j].out[t - jobs[j].outw_before] = 0u;
    }
}

__global__ void __launch_bounds__(256)
batch_gather_kernel(const BatchJobDev *__restrict__ jobs, uint32_t njobs, uint64_t total_groups)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gstride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < total_groups; g += gstride) {
        const uint32_t jb = find_job(jobs, njobs, g, true);
        const BatchJobDev &J = jobs[jb];
        const uint64_t local = g - J.groups_before;
        const uint32_t gpr = J.w_pad >> 5;
        const uint32_t j = (uint32_t)(local / gpr), w0 = (uint32_t)(local % gpr) * 32u;
        if (J.perm && J.padded) gather_group<false, true>(J.in, J.perm, J.s, J.w_pad, j, w0, lane, J.arev);
        else if (J.perm) gather_group<false>(J.in, J.perm, J.s, J.w_pad, j, w0, lane, J.arev);
        else gather_group<true>(J.in, J.perm, J.s, J.w_pad, j, w0, lane, J.arev);
    }
}

__global__ void __launch_bounds__(kHashThreads, 1)
batch_hash_kernel(const BatchJobDev *__restrict__ jobs, const BatchTileDev *__restrict__ tiles, uint32_t ntiles,
                  uint32_t *counter)
{
    __shared__ __align__(16) uint32_t a_s[32 * kHashWC];
    __shared__ __align__(16) uint32_t s_s[kSeedSmemWords];
    __shared__ uint32_t next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t ti = next;
        __syncthreads();
        if (ti >= ntiles) break;
        const BatchTileDev t = tiles[ti];
        const BatchJobDev &J = jobs[t.job];
        const uint32_t *sd = J.seed + (size_t)(J.seed_stride ? t.j0 : 0u) * J.seed_stride + (t.r0 >> 5);
#define EX_RUN_TILE(Q_, J_) \
    hash_tile<Q_, J_>(sd, J.arev, J.w_pad, J.m, J.k, t.r0, t.j0, t.c_begin, t.c_end, J.out, a_s, s_s)
        EX_FOR_VARIANT(t.variant, EX_RUN_TILE)
#undef EX_RUN_TILE
    }
}

// ---- autotuner: GPU time per (CTA, word chunk) of each variant -------------
struct TuneTable {
    bool valid = false;
    double ns_per_chunk[kNumVariants] = {};
};
std::mutex g_tune_mu;
TuneTable g_tune[64];

int measure_variants(int dev, int sms, TuneTable &tt)
{
    // one synthetic job big enough for every variant's tile (k = the tallest
    // tile, m = the widest) so all reads stay inside its buffers
    constexpr uint32_t kM = 32, kChunks = 8, kW = kChunks * kHashWC, kK = kHashWarps * 32 * kMaxQ;
    const uint32_t stride = kK / 32 + kW + 8;
    const uint32_t ntiles = (uint32_t)sms * 3;
    uint32_t *arev = nullptr, *seed = nullptr, *out = nullptr, *counter = nullptr;
    BatchJobDev *djob = nullptr;
    BatchTileDev *dtiles = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = EXTRACT_OK;
    do {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_error(e, "tune stream"); break; }
        if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) { rc = cuda_error(e, "tune events"); break; }
        if ((e = cudaMalloc(&arev, (size_t)kM * kW * 4)) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        if ((e = cudaMalloc(&seed, (size_t)stride * 4)) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        if ((e = cudaMalloc(&out, (size_t)kM * kK / 8)) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        if ((e = cudaMalloc(&counter, 4)) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        if ((e = cudaMalloc(&djob, sizeof(BatchJobDev))) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        if ((e = cudaMalloc(&dtiles, sizeof(BatchTileDev) * ntiles)) != cudaSuccess) { rc = cuda_error(e, "tune alloc"); break; }
        cudaMemsetAsync(arev, 0x5a, (size_t)kM * kW * 4, st);
        cudaMemsetAsync(seed, 0xa5, (size_t)stride * 4, st);
        BatchJobDev hj{};
        hj.seed = seed; hj.arev = arev; hj.out = out; hj.m = kM; hj.k = kK; hj.s = kW * 32; hj.w_pad = kW;
        cudaMemcpyAsync(djob, &hj, sizeof(hj), cudaMemcpyHostToDevice, st);
        std::vector<BatchTileDev> ht(ntiles);
        for (int v = 0; v < kNumVariants && rc == EXTRACT_OK; ++v) {
            for (uint32_t t = 0; t < ntiles; ++t) ht[t] = BatchTileDev{0u, (uint32_t)v, 0u, 0u, 0u, kChunks};
            cudaMemcpyAsync(dtiles, ht.data(), sizeof(BatchTileDev) * ntiles, cudaMemcpyHostToDevice, st);
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaMemsetAsync(counter, 0, 4, st);
                cudaEventRecord(e0, st);
                batch_hash_kernel<<<sms, kHashThreads, 0, st>>>(djob, dtiles, ntiles, counter);
                cudaEventRecord(e1, st);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_error(e, "tune run"); break; }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best = std::min(best, ms);
            }
            tt.ns_per_chunk[v] = (double)best * 1e6 / ((double)ntiles * kChunks);
        }
        if (rc == EXTRACT_OK && (e = cudaGetLastError()) != cudaSuccess) rc = cuda_error(e, "tune");
    } while (0);
    cudaFree(arev); cudaFree(seed); cudaFree(out); cudaFree(counter); cudaFree(djob); cudaFree(dtiles);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    tt.valid = (rc == EXTRACT_OK);
    (void)dev;
    return rc;
}

int tune_table_locked(int dev, int sms, const TuneTable **out)
{
    if (dev < 0 || dev >= 64) return set_error(EXTRACT_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (!g_tune[dev].valid)
        if (int rc = measure_variants(dev, sms, g_tune[dev])) return rc;
    *out = &g_tune[dev];
    return EXTRACT_OK;
}

}  // namespace

int tile_costs(int dev, int sms, const double **ns_per_chunk)
{
    const TuneTable *tt = nullptr;
    if (int rc = tune_table_locked(dev, sms, &tt)) return rc;
    *ns_per_chunk = tt->ns_per_chunk;
    return EXTRACT_OK;
}

int choose_variant(uint32_t m, uint32_t k, uint32_t w_pad, bool per_sub, const double *ns_per_chunk)
{
    const uint32_t nchunks = w_pad / kWordChunk;
    double best = 1e300;
    int pick = variant_id(4, 1);
    for (int v = 0; v < kNumVariants; ++v) {
        if (per_sub && variant_j(v) != 1) continue;
        const double tiles = (double)ceil_div(k, (uint64_t)kHashWarps * 32 * variant_q(v)) *
                             (double)ceil_div(m, (uint64_t)variant_j(v));
        const double t = tiles * nchunks * ns_per_chunk[v];
        if (t < best) { best = t; pick = v; }
    }
    return pick;
}

int launch_batch_hash(const BatchJobDev *jobs, const BatchTileDev *tiles, uint32_t ntiles, uint32_t *counter,
                      int sms, cudaStream_t st)
{
    batch_hash_kernel<<<sms, kHashThreads, 0, st>>>(jobs, tiles, ntiles, counter);
    EX_LAUNCH("batch_hash_kernel");
    return EXTRACT_OK;
}

namespace {

struct BatchJobHost {
    uint64_t n;
    uint32_t m, s, k, flags;
    uint32_t w_pad, variant, seed_stride, nseeds, cps;
    HashPlan plain_plan;  // the single-block heuristic plan (one launch per block)
    uint32_t *perm = nullptr, *arev = nullptr, *seed = nullptr;
    NttPlan *ntt = nullptr;  // set when this job is hashed by the NTT method
    bool tc = false;         // hashed by the tensor-core product (on a lane, like NTT jobs)
    int table_index = -1;    // row of the device job table (direct-method jobs)
    int lane = -1;           // lane of an NTT-method or tensor-core job
};

// NTT and tensor-core jobs run on a few concurrent lanes (stream + NTT work
// buffer each), so small transforms fill the GPU together; jobs are
// assigned longest first to the least loaded lane.
constexpr int kNttLanes = 4;
constexpr uint32_t kTcBatchChunk = 32;  // K blocks of 128 per parity read-back (4096 K)
struct NttLane {
    cudaStream_t st = nullptr;
    uint32_t *work = nullptr;
    cudaEvent_t join = nullptr;
    double load_ns = 0;
};

}  // namespace
}  // namespace ex

using namespace ex;

struct extract_batch {
    int device = 0, num_sms = 0;
    uint32_t flags = 0;
    std::vector<BatchJobHost> jobs;
    std::vector<BatchJobDev> table;  // host copy of the device job table
    BatchJobDev *d_jobs = nullptr;
    BatchTileDev *d_tiles = nullptr;
    uint32_t ntiles = 0;
    uint32_t *d_counter = nullptr;
    uint64_t total_groups = 0, total_out_words = 0;
    double predicted_ms = 0;
    uint32_t ndirect = 0, nntt = 0, ntc = 0;
    uint32_t *d_err = nullptr;  // error word of the tensor-core kernels
    NttLane lanes[kNttLanes];      // concurrent with the persistent launch
    std::vector<uint32_t> ntt_order;  // NTT jobs, longest predicted first
    cudaEvent_t ev_fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string desc;
};

namespace {

void free_batch(extract_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &j : b->jobs) {
        cudaFree(j.perm);
        cudaFree(j.arev);
        cudaFree(j.seed);
        ntt_destroy(j.ntt);
    }
    for (NttLane &L : b->lanes) {
        cudaFree(L.work);
        if (L.join) cudaEventDestroy(L.join);
        if (L.st) cudaStreamDestroy(L.st);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaFree(b->d_err);
    cudaFree(b->d_jobs);
    cudaFree(b->d_tiles);
    cudaFree(b->d_counter);
    delete b;
}

void realign(const uint32_t *src, uint64_t src_words, uint64_t off, uint64_t len, uint32_t *dst, uint64_t dst_words)
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

int launch_batch(extract_batch *b, cudaStream_t st)
{
    const uint32_t nj = b->ndirect;
    if (nj == 0) return EXTRACT_OK;
    const uint32_t zgrid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(b->total_out_words, 256),
                                                                             (uint64_t)b->num_sms * 8));
    batch_zero_kernel<<<zgrid, 256, 0, st>>>(b->d_jobs, nj, b->total_out_words, b->d_counter);
    const uint32_t ggrid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(b->total_groups, 8),
                                                                             (uint64_t)b->num_sms * 64));
    batch_gather_kernel<<<ggrid, 256, 0, st>>>(b->d_jobs, nj, b->total_groups);
    batch_hash_kernel<<<b->num_sms, kHashThreads, 0, st>>>(b->d_jobs, b->d_tiles, b->ntiles, b->d_counter);
    EX_LAUNCH("batch kernels");
    return EXTRACT_OK;
}

}  // namespace

extern "C" {

int extract_batch_create(extract_batch **out, const extract_job_desc *jobs, uint32_t njobs, uint32_t flags)
{
    if (!out) return set_error(EXTRACT_EINVAL, "out is null");
    *out = nullptr;
    if (!jobs || njobs == 0) return set_error(EXTRACT_EINVAL, "empty job list");
    if (flags & ~(EXTRACT_BATCH_NO_GRAPH | EXTRACT_BATCH_NO_TUNE | EXTRACT_BATCH_DIRECT_ONLY | EXTRACT_BATCH_TENSOR))
        return set_error(EXTRACT_EINVAL, "unknown batch flags 0x%x", flags);
    if ((flags & EXTRACT_BATCH_DIRECT_ONLY) && (flags & EXTRACT_BATCH_TENSOR))
        return set_error(EXTRACT_EINVAL, "EXTRACT_BATCH_DIRECT_ONLY and EXTRACT_BATCH_TENSOR are exclusive");
    const uint32_t known = EXTRACT_SEED_PER_SUBBLOCK | EXTRACT_IDENTITY_PERM | EXTRACT_SAMPLING_IID | (0x3fu << 8);
    for (uint32_t i = 0; i < njobs; ++i) {
        const extract_job_desc &d = jobs[i];
        if (!d.seed_bits_host) return set_error(EXTRACT_EINVAL, "job %u: null seed", i);
        if (d.flags & ~known) return set_error(EXTRACT_EINVAL, "job %u: unknown flags 0x%x", i, d.flags);
        const bool iid = (d.flags & EXTRACT_SAMPLING_IID) != 0;
        if (d.m < 1 || d.s < 1 || d.k < 1 || d.k > d.s || d.n > (1ull << 32) || (!iid && (uint64_t)d.m * d.s > d.n))
            return set_error(EXTRACT_EINVAL, "job %u: bad shape n=%llu m=%u s=%u k=%u", i,
                             (unsigned long long)d.n, d.m, d.s, d.k);
        if (iid && ((d.flags & EXTRACT_IDENTITY_PERM) || d.n >= (1ull << 32) || d.m > (1u << 16)))
            return set_error(EXTRACT_EINVAL, "job %u: the i.i.d. law needs n < 2^32, m <= 2^16, no identity order", i);
    }
    extract_batch *b = new (std::nothrow) extract_batch();
    if (!b) return set_error(EXTRACT_ENOMEM, "host allocation failed");
    b->flags = flags;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) { delete b; return cuda_error(e, "device query"); }

    const TuneTable *tt = nullptr;
    TuneTable untuned;
    if (!(flags & EXTRACT_BATCH_NO_TUNE)) {
        if (int rc = tune_table_locked(b->device, b->num_sms, &tt)) { delete b; return rc; }
    } else {
        for (int v = 0; v < kNumVariants; ++v) untuned.ns_per_chunk[v] = 1.0;
        tt = &untuned;
    }

    // per-job plan: variant with the least predicted time
    b->jobs.resize(njobs);
    double total_ns = 0;
    for (uint32_t i = 0; i < njobs; ++i) {
        const extract_job_desc &d = jobs[i];
        BatchJobHost &J = b->jobs[i];
        J.n = d.n; J.m = d.m; J.s = d.s; J.k = d.k; J.flags = d.flags;
        J.w_pad = (uint32_t)round_up(ceil_div(d.s, 32), kWordChunk);
        const bool per_sub = (d.flags & EXTRACT_SEED_PER_SUBBLOCK) != 0;
        J.plain_plan = plan_hash(d.m, d.k, J.w_pad, per_sub, b->num_sms);
        const uint32_t nchunks = J.w_pad / kWordChunk;
        if (flags & EXTRACT_BATCH_NO_TUNE)
            J.variant = (uint32_t)J.plain_plan.variant;
        else
            J.variant = (uint32_t)choose_variant(d.m, d.k, J.w_pad, per_sub, tt->ns_per_chunk);
        const uint64_t tiles = ceil_div(d.k, (uint64_t)kHashWarps * 32 * variant_q(J.variant)) *
                               ceil_div(d.m, (uint64_t)variant_j(J.variant));
        const double direct_ns = (double)tiles * nchunks * tt->ns_per_chunk[J.variant];
        // the least predicted time of the three methods (tensor cores only
        // with a shared seed; the direct kernel only with DIRECT_ONLY)
        const bool any = !(flags & EXTRACT_BATCH_DIRECT_ONLY);
        const double ntt_ns = any && ntt_shape(d.s, d.k, -1, per_sub).N != 0
                                  ? predict_ntt_s(d.m, d.s, d.k, -1, per_sub) * 1e9 : 1e300;
        const double tc_ns = any && !per_sub ? predict_tc_s(d.m, d.k, d.s) * 1e9 : 1e300;
        if ((flags & EXTRACT_BATCH_TENSOR) && !per_sub) {
            J.table_index = -2;  // marks a lane job until its plan exists
            J.tc = true;
        } else if (std::min(ntt_ns, tc_ns) < direct_ns) {
            J.table_index = -2;
            J.tc = tc_ns < ntt_ns;
        } else {
            total_ns += direct_ns;
        }
        HashPlan vp;
        vp.q = variant_q(J.variant); vp.j = variant_j(J.variant);
        vp.gx = (uint32_t)ceil_div(d.k, vp.rows());
        J.seed_stride = std::max(seed_stride_words(vp, d.k, J.w_pad), seed_stride_words(J.plain_plan, d.k, J.w_pad));
        J.nseeds = per_sub ? d.m : 1u;
    }
    b->predicted_ms = total_ns / 1e6;  // costs are whole-GPU time per CTA-chunk
    // split word ranges so no tile exceeds ~1/8 of an SM's share of the batch
    const double tile_cap_ns = std::max(1.0, total_ns / ((double)b->num_sms * 8.0));
    std::vector<std::pair<double, BatchTileDev>> tl;
    for (uint32_t i = 0; i < njobs; ++i) {
        BatchJobHost &J = b->jobs[i];
        if (J.table_index == -2) {
            ++(J.tc ? b->ntc : b->nntt);
            continue;
        }
        J.table_index = (int)b->ndirect++;
        const uint32_t nchunks = J.w_pad / kWordChunk;
        const double cost = tt->ns_per_chunk[J.variant];
        J.cps = (uint32_t)std::max<double>(1.0, std::min<double>((double)nchunks, tile_cap_ns / cost));
        const uint32_t rows = (uint32_t)kHashWarps * 32u * (uint32_t)variant_q(J.variant);
        const uint32_t gx = (uint32_t)ceil_div(J.k, rows), gy = (uint32_t)ceil_div(J.m, (uint32_t)variant_j(J.variant));
        for (uint32_t by = 0; by < gy; ++by)
            for (uint32_t bx = 0; bx < gx; ++bx)
                for (uint32_t c = 0; c < nchunks; c += J.cps) {
                    const uint32_t ce = std::min(nchunks, c + J.cps);
                    tl.push_back({(ce - c) * cost, BatchTileDev{(uint32_t)J.table_index, J.variant, bx * rows,
                                                                by * (uint32_t)variant_j(J.variant), c, ce}});
                }
    }
    std::stable_sort(tl.begin(), tl.end(), [](const auto &a, const auto &c) { return a.first > c.first; });
    if (tl.size() >= (1ull << 32)) { delete b; return set_error(EXTRACT_EINVAL, "too many tiles"); }
    b->ntiles = (uint32_t)tl.size();

    int rc = EXTRACT_OK;
    cudaStream_t st = nullptr;
    do {
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_error(e, "stream"); break; }
        b->table.resize(b->ndirect);
        uint64_t groups = 0, outw = 0, work = 0;
        std::vector<std::pair<double, uint32_t>> nj_cost;
        for (uint32_t i = 0; i < njobs; ++i)
            if (b->jobs[i].table_index == -2) {
                const bool ps = (jobs[i].flags & EXTRACT_SEED_PER_SUBBLOCK) != 0;
                if (b->jobs[i].tc) {
                    nj_cost.push_back({predict_tc_s(jobs[i].m, jobs[i].k, jobs[i].s), i});
                } else {
                    work = std::max(work, ntt_work_words(jobs[i].m, jobs[i].s, jobs[i].k, -1, ps));
                    nj_cost.push_back({predict_ntt_s(jobs[i].m, jobs[i].s, jobs[i].k, -1, ps), i});
                }
            }
        std::stable_sort(nj_cost.begin(), nj_cost.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
        const int nlanes = (int)std::min<size_t>(kNttLanes, nj_cost.size());
        for (auto &c : nj_cost) {  // longest first onto the least loaded lane
            int best = 0;
            for (int l = 1; l < nlanes; ++l)
                if (b->lanes[l].load_ns < b->lanes[best].load_ns) best = l;
            b->lanes[best].load_ns += c.first;
            b->jobs[c.second].lane = best;
            b->ntt_order.push_back(c.second);
        }
        for (int l = 0; l < nlanes && rc == EXTRACT_OK; ++l) {
            NttLane &L = b->lanes[l];
            if (work && (e = cudaMalloc(&L.work, work * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(ntt work)"); break; }
            if ((e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming)) != cudaSuccess) {
                rc = cuda_error(e, "ntt lane");
                break;
            }
        }
        if (rc != EXTRACT_OK) break;
        if (nlanes && (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
            rc = cuda_error(e, "ntt fork event");
            break;
        }
        if (b->ntc && ((e = cudaMalloc(&b->d_err, 4)) != cudaSuccess || (e = cudaMemset(b->d_err, 0, 4)) != cudaSuccess)) {
            rc = cuda_error(e, "tensor-core error word");
            break;
        }
        for (uint32_t i = 0; i < njobs && rc == EXTRACT_OK; ++i) {
            const extract_job_desc &d = jobs[i];
            BatchJobHost &J = b->jobs[i];
            const uint64_t L = (uint64_t)d.s + d.k - 1;
            std::vector<uint32_t> host((size_t)J.nseeds * J.seed_stride);
            const uint64_t src_words = ceil_div(L * J.nseeds, 32);
            for (uint32_t q = 0; q < J.nseeds; ++q)
                realign(d.seed_bits_host, src_words, (uint64_t)q * L, L, host.data() + (size_t)q * J.seed_stride,
                        J.seed_stride);
            if ((e = cudaMalloc(&J.seed, host.size() * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(seed)"); break; }
            if ((e = cudaMemcpy(J.seed, host.data(), host.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) { rc = cuda_error(e, "seed copy"); break; }
            if ((e = cudaMalloc(&J.arev, (size_t)d.m * J.w_pad * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(sub-blocks)"); break; }
            if (!(d.flags & EXTRACT_IDENTITY_PERM)) {
                const bool iid = (d.flags & EXTRACT_SAMPLING_IID) != 0;
                const uint64_t len = iid ? (uint64_t)d.m * d.s : d.n;
                if ((e = cudaMalloc(&J.perm, (size_t)std::max<uint64_t>(len, 1) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(order)"); break; }
                const uint32_t kb = (d.flags >> 8) & 0x3fu;
                const uint64_t mask = kb ? ~((1ull << (64u - kb)) - 1ull) : ~0ull;
                if (iid) {
                    std::vector<uint64_t> sizes;
                    if ((rc = build_iid_order(d.n, d.sampling_key, mask, d.m, d.s, J.perm, &sizes, st, b->num_sms)) !=
                        EXTRACT_OK) {
                        if (rc == EXTRACT_EABORT) {
                            const std::string why = extract_last_error();
                            rc = set_error(EXTRACT_EABORT, "job %u: %s", i, why.c_str());
                        }
                        break;
                    }
                } else if ((rc = build_perm(d.n, d.sampling_key, mask, J.perm, st, b->num_sms)) != EXTRACT_OK) {
                    break;
                }
            }
            if (J.table_index == -2) {
                if (!J.tc && (rc = ntt_create(&J.ntt, d.m, d.s, d.k, J.seed, st, b->lanes[J.lane].work, -1,
                                              J.nseeds > 1 ? J.seed_stride : 0)) != EXTRACT_OK)
                    break;
                continue;
            }
            BatchJobDev &T = b->table[J.table_index];
            T.perm = J.perm; T.in = nullptr; T.out = nullptr; T.seed = J.seed; T.arev = J.arev;
            T.groups_before = groups; T.outw_before = outw;
            T.seed_stride = J.nseeds > 1 ? J.seed_stride : 0u;
            T.m = d.m; T.s = d.s; T.k = d.k; T.w_pad = J.w_pad;
            T.padded = (d.flags & EXTRACT_SAMPLING_IID) ? 1u : 0u;
            groups += (uint64_t)d.m * (J.w_pad / 32);
            outw += ceil_div((uint64_t)d.m * d.k, 32);
        }
        if (rc != EXTRACT_OK) break;
        b->total_groups = groups;
        b->total_out_words = outw;
        if ((e = cudaMalloc(&b->d_jobs, sizeof(BatchJobDev) * std::max<uint32_t>(1, b->ndirect))) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(jobs)"); break; }
        if ((e = cudaMalloc(&b->d_tiles, sizeof(BatchTileDev) * std::max<size_t>(1, tl.size()))) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(tiles)"); break; }
        if ((e = cudaMalloc(&b->d_counter, 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(counter)"); break; }
        std::vector<BatchTileDev> ht(tl.size());
        for (size_t t = 0; t < tl.size(); ++t) ht[t] = tl[t].second;
        if ((e = cudaMemcpy(b->d_tiles, ht.data(), sizeof(BatchTileDev) * ht.size(), cudaMemcpyHostToDevice)) != cudaSuccess) { rc = cuda_error(e, "tiles copy"); break; }
        if (b->ndirect &&
            (e = cudaMemcpy(b->d_jobs, b->table.data(), sizeof(BatchJobDev) * b->ndirect, cudaMemcpyHostToDevice)) != cudaSuccess) { rc = cuda_error(e, "jobs copy"); break; }
        if (b->ndirect && !(flags & EXTRACT_BATCH_NO_GRAPH)) {
            if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) { rc = cuda_error(e, "capture"); break; }
            int lrc = launch_batch(b, st);
            e = cudaStreamEndCapture(st, &b->graph);
            if (lrc != EXTRACT_OK) { rc = lrc; break; }
            if (e != cudaSuccess) { rc = cuda_error(e, "end capture"); break; }
            if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) { rc = cuda_error(e, "graph instantiate"); break; }
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "batch create"); break; }
    } while (0);
    if (st) cudaStreamDestroy(st);
    if (rc != EXTRACT_OK) { free_batch(b); return rc; }

    int counts[kNumVariants] = {};
    for (auto &J : b->jobs)
        if (J.table_index >= 0) counts[J.variant]++;
    char buf[1024];
    int len = snprintf(buf, sizeof(buf),
                       "batch: %u jobs (%u NTT and %u tensor-core on concurrent lanes, %u direct), %u tiles, graph=%s, "
                       "tuned=%s, direct part predicted %.3f ms; variants",
                       njobs, b->nntt, b->ntc, b->ndirect, b->ntiles, b->exec ? "yes" : "no",
                       (flags & EXTRACT_BATCH_NO_TUNE) ? "no" : "yes", b->predicted_ms);
    for (int v = 0; v < kNumVariants && len < (int)sizeof(buf) - 64; ++v)
        if (counts[v])
            len += snprintf(buf + len, sizeof(buf) - len, " q%d/j%d:%d(%.1fns/chunk)", variant_q(v), variant_j(v),
                            counts[v], tt->ns_per_chunk[v]);
    b->desc = buf;
    *out = b;
    return EXTRACT_OK;
}

int extract_batch_run(extract_batch *b, void *stream, const uint32_t *const *in_bits_dev,
                      uint32_t *const *out_bits_dev)
{
    if (!b) return set_error(EXTRACT_EINVAL, "null batch");
    if (!in_bits_dev || !out_bits_dev) return set_error(EXTRACT_EINVAL, "null pointer arrays");
    const size_t nj = b->jobs.size();
    for (size_t i = 0; i < nj; ++i) {
        if (!in_bits_dev[i] || !out_bits_dev[i]) return set_error(EXTRACT_EINVAL, "job %zu: null buffer", i);
        const int t = b->jobs[i].table_index;
        if (t >= 0) {
            b->table[t].in = in_bits_dev[i];
            b->table[t].out = out_bits_dev[i];
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    // NTT and tensor-core jobs: forked onto the batch's lanes (each lane's
    // jobs one after another on its stream and work buffer), concurrent with
    // the persistent launch below
    if (b->nntt + b->ntc) {
        EX_CUDA(cudaEventRecord(b->ev_fork, st));
        for (NttLane &L : b->lanes)
            if (L.st) EX_CUDA(cudaStreamWaitEvent(L.st, b->ev_fork, 0));
        for (uint32_t i : b->ntt_order) {
            const BatchJobHost &J = b->jobs[i];
            const NttLane &L = b->lanes[J.lane];
            if (int rc = launch_gather(in_bits_dev[i], J.perm, J.m, J.s, J.w_pad, J.arev, L.st, b->num_sms, 0,
                                       (J.flags & EXTRACT_SAMPLING_IID) != 0, J.n))
                return rc;
            if (J.tc) {
                if (int rc = launch_hash_tc(J.seed, J.seed_stride, J.arev, J.w_pad, J.m, J.s, J.k, out_bits_dev[i],
                                            b->d_err, L.st, kTcBatchChunk))
                    return rc;
            } else if (int rc = ntt_hash(J.ntt, J.arev, J.w_pad, J.m, J.s, J.k, out_bits_dev[i], L.st, L.work)) {
                return rc;
            }
        }
        for (NttLane &L : b->lanes)
            if (L.st) EX_CUDA(cudaEventRecord(L.join, L.st));
    }
    if (b->ndirect) {
        // pageable source: the copy is staged before the call returns, so the
        // host table can be rewritten by the next run at once
        EX_CUDA(cudaMemcpyAsync(b->d_jobs, b->table.data(), sizeof(BatchJobDev) * b->ndirect, cudaMemcpyHostToDevice,
                                st));
        if (b->exec) {
            EX_CUDA(cudaGraphLaunch(b->exec, st));
        } else if (int rc = launch_batch(b, st)) {
            return rc;
        }
    }
    for (NttLane &L : b->lanes)
        if (L.st) EX_CUDA(cudaStreamWaitEvent(st, L.join, 0));
    return EXTRACT_OK;
}

int extract_batch_run_sequential(extract_batch *b, void *stream, const uint32_t *const *in_bits_dev,
                                 uint32_t *const *out_bits_dev)
{
    if (!b) return set_error(EXTRACT_EINVAL, "null batch");
    if (!in_bits_dev || !out_bits_dev) return set_error(EXTRACT_EINVAL, "null pointer arrays");
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        const BatchJobHost &J = b->jobs[i];
        if (!in_bits_dev[i] || !out_bits_dev[i]) return set_error(EXTRACT_EINVAL, "job %zu: null buffer", i);
        if (int rc = launch_gather(in_bits_dev[i], J.perm, J.m, J.s, J.w_pad, J.arev, st, b->num_sms, 0,
                                   (J.flags & EXTRACT_SAMPLING_IID) != 0, J.n))
            return rc;
        if (J.ntt) {
            if (int rc = ntt_hash(J.ntt, J.arev, J.w_pad, J.m, J.s, J.k, out_bits_dev[i], st)) return rc;
        } else if (J.tc) {
            if (int rc = launch_hash_tc(J.seed, J.seed_stride, J.arev, J.w_pad, J.m, J.s, J.k, out_bits_dev[i],
                                        b->d_err, st, kTcBatchChunk))
                return rc;
        } else if (int rc = launch_hash(J.plain_plan, J.seed, J.nseeds > 1 ? J.seed_stride : 0u, J.arev, J.w_pad,
                                        J.m, J.k, out_bits_dev[i], st)) {
            return rc;
        }
    }
    return EXTRACT_OK;
}

int extract_batch_status(extract_batch *b)
{
    if (!b) return set_error(EXTRACT_EINVAL, "null batch");
    int rc = EXTRACT_OK;
    for (const BatchJobHost &J : b->jobs)  // every plan's word is read and cleared
        if (J.ntt)
            if (int r = ntt_status(J.ntt)) rc = r;
    if (rc) return rc;
    if (!b->d_err) return EXTRACT_OK;
    uint32_t v = 0;
    EX_CUDA(cudaDeviceSynchronize());
    EX_CUDA(cudaMemcpy(&v, b->d_err, 4, cudaMemcpyDeviceToHost));
    if (!v) return EXTRACT_OK;
    EX_CUDA(cudaMemset(b->d_err, 0, 4));
    return set_error(EXTRACT_ETIMEDOUT, "a tensor-core hash kernel of the batch gave up waiting for its multiplies");
}

int extract_batch_describe(extract_batch *b, char *buf, uint32_t buflen)
{
    if (!b) return set_error(EXTRACT_EINVAL, "null batch");
    if (!buf || !buflen) return set_error(EXTRACT_EINVAL, "empty buffer");
    snprintf(buf, buflen, "%s", b->desc.c_str());
    return EXTRACT_OK;
}

int extract_batch_destroy(extract_batch *b)
{
    if (!b) return EXTRACT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(b);
    if (e != cudaSuccess) return cuda_error(e, "batch destroy");
    return EXTRACT_OK;
}

}  // extern "C"
