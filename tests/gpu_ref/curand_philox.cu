// Prints cuRAND's Philox4x32-10 device outputs (test reference only).
// Usage: curand_philox <seed> <subsequence> <n_blocks>
// For each of n_blocks consecutive curand4() calls after
// curand_init(seed, subsequence, 0, &state) one line "x y z w" (decimal).
#include <cstdio>
#include <cstdlib>
#include <curand_kernel.h>

__global__ void draw(unsigned long long seed, unsigned long long subseq, int n, uint4 *out)
{
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, 0ull, &st);
    for (int i = 0; i < n; ++i) out[i] = curand4(&st);
}

int main(int argc, char **argv)
{
    if (argc < 4) return 2;
    const unsigned long long seed = strtoull(argv[1], nullptr, 10);
    const unsigned long long sub = strtoull(argv[2], nullptr, 10);
    const int n = atoi(argv[3]);
    if (n <= 0 || n > 4096) return 2;
    uint4 *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(uint4)) != cudaSuccess) return 3;
    draw<<<1, 1>>>(seed, sub, n, d);
    uint4 *h = (uint4 *)malloc(n * sizeof(uint4));
    if (cudaMemcpy(h, d, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    for (int i = 0; i < n; ++i) printf("%u %u %u %u\n", h[i].x, h[i].y, h[i].z, h[i].w);
    cudaFree(d);
    free(h);
    return 0;
}
