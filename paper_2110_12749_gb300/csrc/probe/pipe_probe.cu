// Throughput probes of the integer, FP32 and shared-load pipes of one GPU: the
// basis of the integer-issue roofline of the dedispersion kernel.  Two CTAs of
// 512 threads per SM, 8 independent dependency chains per thread, SM cycles
// from clock64 inside each CTA; throughput in lane-ops per clock per SM.
// Shared loads are volatile and move every iteration, so that the compiler
// keeps every one of them.  Not part of libgsp: built and run by
// paper_2110_12749_gb300.build.run_pipe_probe().
#include <cstdio>
#include <cstdint>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("ERR %s %s\n", #x, cudaGetErrorString(e)); return 1; } } while (0)

constexpr int ITERS = 4096;
constexpr int CH = 8;

template <int OP>
__global__ void __launch_bounds__(512, 2) probe(uint32_t seed, uint32_t one, uint32_t *out, long long *cyc) {
    __shared__ __align__(16) uint32_t sm[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) sm[i] = i * 2654435761u + seed;
    __syncthreads();
    uint32_t a[CH];
    float f[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) { a[c] = seed + c * 7 + threadIdx.x; f[c] = (float)(a[c] & 255); }
    uint32_t b = seed ^ 0x1234567u, d = seed * 3u + 1;
    uint32_t addr = (uint32_t)__cvta_generic_to_shared(sm) + 4 * (threadIdx.x & 31);
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            if (OP == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(b));                 // IADD
            if (OP == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d)); // LOP3
            if (OP == 2) asm volatile("prmt.b32 %0, %0, %1, 0x4341;" : "+r"(a[c]) : "r"(b));       // PRMT
            if (OP == 3) asm volatile("shf.l.wrap.b32 %0, %0, %1, 3;" : "+r"(a[c]) : "r"(b));      // SHF
            if (OP == 4) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(one), "r"(b)); // IMAD
            if (OP == 5) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(b), "r"(d)); // IMAD.HI
            if (OP == 6) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(1.0f), "f"(0.5f)); // FFMA
            if (OP == 7) { uint32_t v; asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr + 128 * c + ((it & 7) << 10))); a[c] += v; } // LDS + add
            if (OP == 8) {
                // the dedispersion accumulation mix per two words: 2 LDS, 2 PRMT, 1 IADD3, 2 IMAD
                uint32_t w1, w2;
                asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(w1) : "r"(addr + 256 * (c & 3) + ((it & 7) << 10)));
                asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(w2) : "r"(addr + 256 * (c & 3) + 128 + ((it & 7) << 10)));
                uint32_t o1, o2;
                asm volatile("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(o1) : "r"(w1));
                asm volatile("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(o2) : "r"(w2));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(w1 + w2));
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(d) : "r"(o1), "r"(one));
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(b) : "r"(o2), "r"(one));
            }
            if (OP == 10) {
                // 16-byte shared loads: bytes per clock (one IMAD per load keeps the value live)
                uint32_t x, y, z, w;
                asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                             : "r"(addr * 4 - 3 * (uint32_t)__cvta_generic_to_shared(sm) + 512 * (c & 3) + ((it & 3) << 11)));
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(a[c]) : "r"(x ^ y ^ z ^ w), "r"(one));
            }
            if (OP == 11) {
                // packed FP32 FMA: two independent FMAs per instruction (f[c], f[c ^ 1] as a pair)
                if ((c & 1) == 0) {
                    uint64_t pr = ((uint64_t)__float_as_uint(f[c + 1]) << 32) | __float_as_uint(f[c]);
                    const uint64_t m2 = 0x3f8000003f800000ull, c2 = 0x3f0000003f000000ull;  // (1, 1), (0.5, 0.5)
                    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(pr) : "l"(m2), "l"(c2));
                    f[c] = __uint_as_float((uint32_t)pr);
                    f[c + 1] = __uint_as_float((uint32_t)(pr >> 32));
                }
            }
            if (OP == 9) {
                // the same mix without the shared loads (register operands only)
                uint32_t w1 = a[c] ^ it, w2 = a[(c + 1) % CH];
                uint32_t o1, o2;
                asm volatile("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(o1) : "r"(w1));
                asm volatile("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(o2) : "r"(w2));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(w1 + w2));
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(d) : "r"(o1), "r"(one));
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(b) : "r"(o2), "r"(one));
            }
        }
    }
    long long t1 = clock64();
    uint32_t s = b ^ d;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= a[c] ^ __float_as_uint(f[c]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int OP>
int run(const char *name, double ops_per_iter_chain, int nsm, uint32_t *out, long long *cyc) {
    const int grid = nsm * 2, block = 512;
    probe<OP><<<grid, block>>>(1, 1, out, cyc);
    CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0);
    probe<OP><<<grid, block>>>(2, 1, out, cyc);
    cudaEventRecord(e1);
    CK(cudaDeviceSynchronize());
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    std::vector<long long> c(grid);
    CK(cudaMemcpy(c.data(), cyc, grid * sizeof(long long), cudaMemcpyDeviceToHost));
    std::sort(c.begin(), c.end());
    double med = (double)c[grid / 2];
    // per SM: two CTAs of 512 threads run together
    double ops_sm = 2.0 * block * (double)ITERS * CH * ops_per_iter_chain;
    double per_clk = ops_sm / med;
    double clk_mhz = med / (ms * 1e3);
    printf("%-28s %8.1f lane-ops/clk/SM   (median CTA %.0f cycles, %.3f ms, implied SM clock %.0f MHz)\n",
           name, per_clk, med, ms, clk_mhz);
    return 0;
}

int main() {
    int dev = 0, nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp pr; cudaGetDeviceProperties(&pr, dev);
    printf("device %s, %d SMs, CC %d.%d\n", pr.name, nsm, pr.major, pr.minor);
    uint32_t *out; long long *cyc;
    CK(cudaMalloc(&out, (size_t)nsm * 2 * 512 * 4));
    CK(cudaMalloc(&cyc, (size_t)nsm * 2 * 8));
    run<0>("add.u32 (IADD3)", 1, nsm, out, cyc);
    run<1>("lop3.b32 (LOP3)", 1, nsm, out, cyc);
    run<2>("prmt.b32 (PRMT)", 1, nsm, out, cyc);
    run<3>("shf.l.wrap (SHF)", 1, nsm, out, cyc);
    run<4>("mad.lo.u32 (IMAD)", 1, nsm, out, cyc);
    run<5>("mad.hi.u32 (IMAD.HI)", 1, nsm, out, cyc);
    run<6>("fma.rn.f32 (FFMA)", 1, nsm, out, cyc);
    run<7>("ld.shared.u32 + add", 1, nsm, out, cyc);
    // OP 8/9: 8 byte-adds per chain step (two 4-byte words)
    run<8>("SWAR mix, byte-adds (LDS)", 8, nsm, out, cyc);
    run<9>("SWAR mix, byte-adds (regs)", 8, nsm, out, cyc);
    run<10>("ld.shared.v4 (bytes)", 16, nsm, out, cyc);
    // OP 11: one fma.rn.f32x2 per two chains, i.e. one FP32 FMA per chain step
    run<11>("fma.rn.f32x2 (FMAs)", 1, nsm, out, cyc);
    printf("done\n");
    return 0;
}
