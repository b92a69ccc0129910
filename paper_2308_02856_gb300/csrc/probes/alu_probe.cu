// Throughput probes for the roofline of the hashing kernels: LOP3 (integer
// ALU), a SHF+LOP3 mix, and the legacy mma.sync paths (b1 and.popc, s8, e4m3)
// that a tensor-core GF(2) formulation could use.  In-bounds, no waits.
// Built and run by paper_2308_02856_gb300.build.run_alu_probe().
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void lop3_probe(uint32_t *out, long long *cyc, uint32_t seed, int iters)
{
    uint32_t a[16], b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) { a[i] = seed * (threadIdx.x + i * 7 + 1); b[i] = seed ^ (i * 0x9e3779b9u + threadIdx.x); }
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] ^= b[i] & a[(i + 5) & 15];
    }
    long long t1 = clock64();
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) r ^= a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// per 4 words: 4 SHF + 32 LOP3 (like a q=1, j=8 tile)
__global__ void shf_lop3_probe(uint32_t *out, long long *cyc, uint32_t seed, int iters)
{
    uint32_t acc[8], s0 = seed + threadIdx.x, s1 = seed * 3u, a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { acc[i] = 0; a[i] = seed * (i + 11u); }
    const int lane = threadIdx.x & 31;
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        uint32_t w = __funnelshift_r(s0, s1, lane);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] ^= w & a[i];
        s0 = s1 ^ acc[it & 7]; s1 = w;
    }
    long long t1 = clock64();
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) r ^= acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void b1mma_probe(uint32_t *out, long long *cyc, uint32_t seed, int iters)
{
    uint32_t a0 = seed ^ threadIdx.x, a1 = seed * 3u, a2 = seed + 7u, a3 = ~seed;
    uint32_t b0 = seed * 5u + threadIdx.x, b1 = seed ^ 0x55u;
    int c[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[u][v] = 0;
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc "
                         "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                         : "+r"(c[u][0]), "+r"(c[u][1]), "+r"(c[u][2]), "+r"(c[u][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    long long t1 = clock64();
    int r = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) r += c[u][0] + c[u][1] + c[u][2] + c[u][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void s8mma_probe(uint32_t *out, long long *cyc, uint32_t seed, int iters)
{
    uint32_t a0 = seed ^ threadIdx.x, a1 = seed * 3u, a2 = seed + 7u, a3 = ~seed;
    uint32_t b0 = seed * 5u + threadIdx.x, b1 = seed ^ 0x55u;
    int c[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[u][v] = 0;
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
                         "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                         : "+r"(c[u][0]), "+r"(c[u][1]), "+r"(c[u][2]), "+r"(c[u][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    long long t1 = clock64();
    int r = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) r += c[u][0] + c[u][1] + c[u][2] + c[u][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void e4m3mma_probe(uint32_t *out, long long *cyc, uint32_t seed, int iters)
{
    uint32_t a0 = 0x38383838u, a1 = 0x38003800u, a2 = 0x00383800u, a3 = 0x38000038u;
    uint32_t b0 = 0x38380038u, b1 = 0x00380038u;
    float c[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[u][v] = 0.f;
    long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 "
                         "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                         : "+f"(c[u][0]), "+f"(c[u][1]), "+f"(c[u][2]), "+f"(c[u][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    long long t1 = clock64();
    float r = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) r += c[u][0] + c[u][1] + c[u][2] + c[u][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

typedef void (*probe_fn)(uint32_t *, long long *, uint32_t, int);

static int run(const char *name, probe_fn f, int sms, int bps, int threads, int iters, double work_per_thread_iter,
               const char *unit, uint32_t *out, long long *cyc)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
    int blocks = sms * bps;
    f<<<blocks, threads>>>(out, cyc, 12345u, iters / 10);
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0));
    f<<<blocks, threads>>>(out, cyc, 12345u, iters);
    CK(cudaEventRecord(e1));
    CK(cudaDeviceSynchronize());
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    long long hc[4096];
    CK(cudaMemcpy(hc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
    double avgc = 0;
    for (int i = 0; i < blocks; ++i) avgc += (double)hc[i];
    avgc /= blocks;
    double total = (double)blocks * threads * iters * work_per_thread_iter;
    double per_sm_clk = total / sms / avgc;  // blocks of one SM run concurrently
    printf("%-10s blocks=%d thr=%d iters=%d: %.3f ms, %.3e %s/s, %.1f %s/clk/SM (avg %.0f cyc/block), implied clock %.0f MHz\n",
           name, blocks, threads, iters, ms, total / (ms * 1e-3), unit, per_sm_clk, unit, avgc,
           avgc / (ms * 1e-3) / 1e6);
    return 0;
}

int main()
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, dev));
    printf("device %s, %d SMs, cc %d.%d\n", p.name, sms, p.major, p.minor);
    uint32_t *out;
    long long *cyc;
    CK(cudaMalloc(&out, sizeof(uint32_t) * 4096 * 1024));
    CK(cudaMalloc(&cyc, sizeof(long long) * 4096));
    for (int rep = 0; rep < 2; ++rep) {
        run("lop3", lop3_probe, sms, 4, 256, 200000, 16, "LOP3", out, cyc);
        run("lop3x8w", lop3_probe, sms, 1, 256, 200000, 16, "LOP3", out, cyc);
        run("shf+lop3", shf_lop3_probe, sms, 4, 256, 200000, 9, "instr", out, cyc);
        // mma: work unit = MMA instructions per warp (per thread-iter x 1/32)
        run("b1mma", b1mma_probe, sms, 4, 256, 20000, 8.0 * 32768 / 32, "bitMAC", out, cyc);
        run("s8mma", s8mma_probe, sms, 4, 256, 20000, 8.0 * 4096 / 32, "MAC", out, cyc);
        run("e4m3mma", e4m3mma_probe, sms, 4, 256, 20000, 8.0 * 4096 / 32, "MAC", out, cyc);
    }
    return 0;
}
