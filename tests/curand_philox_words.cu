// Philox4x32-10 output words from cuRAND's device generator (an
// implementation independent of this repository), for the Philox known-answer
// test.  Reads lines "c0 c1 c2 c3 k0 k1" (hex) from stdin and prints, per
// line, the four words of cuRAND's block function curand_Philox4x32_10 for
// that counter and key, then the four words curand4() returns after
// curand_init(seed, subsequence, offset), or "-" when the counter cannot be
// reached that way.  cuRAND's state for curand_init with an offset that is a
// multiple of 4 has key = (seed low, seed high) and counter = (offset / 4
// low, offset / 4 high, subsequence low, subsequence high), and curand4()
// returns that counter's block; offset = 4 (c0 + 2^32 c1) fits 64 bits when
// c1 < 2^30.
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdio>
#include <vector>

__global__ void k_words(const unsigned* in, unsigned* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned* c = in + 6 * i;
  const uint4 b = curand_Philox4x32_10(make_uint4(c[0], c[1], c[2], c[3]), make_uint2(c[4], c[5]));
  out[8 * i] = b.x;
  out[8 * i + 1] = b.y;
  out[8 * i + 2] = b.z;
  out[8 * i + 3] = b.w;
  if (c[1] < (1u << 30)) {
    const unsigned long long seed = (unsigned long long)c[4] | ((unsigned long long)c[5] << 32);
    const unsigned long long subseq = (unsigned long long)c[2] | ((unsigned long long)c[3] << 32);
    const unsigned long long block = (unsigned long long)c[0] | ((unsigned long long)c[1] << 32);
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, 4ull * block, &st);
    const uint4 w = curand4(&st);
    out[8 * i + 4] = w.x;
    out[8 * i + 5] = w.y;
    out[8 * i + 6] = w.z;
    out[8 * i + 7] = w.w;
  }
}

int main() {
  std::vector<unsigned> in;
  unsigned v[6];
  while (std::scanf("%x %x %x %x %x %x", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6)
    for (int k = 0; k < 6; ++k) in.push_back(v[k]);
  const int n = (int)(in.size() / 6);
  if (n == 0) return 2;
  unsigned *d_in = nullptr, *d_out = nullptr;
  if (cudaMalloc(&d_in, in.size() * 4) != cudaSuccess || cudaMalloc(&d_out, (size_t)n * 32) != cudaSuccess) return 3;
  cudaMemcpy(d_in, in.data(), in.size() * 4, cudaMemcpyHostToDevice);
  k_words<<<(n + 127) / 128, 128>>>(d_in, d_out, n);
  std::vector<unsigned> out((size_t)n * 8);
  if (cudaMemcpy(out.data(), d_out, out.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
  for (int i = 0; i < n; ++i) {
    const unsigned* o = out.data() + 8 * (size_t)i;
    std::printf("%08x %08x %08x %08x", o[0], o[1], o[2], o[3]);
    if (in[6 * (size_t)i + 1] < (1u << 30)) std::printf(" %08x %08x %08x %08x\n", o[4], o[5], o[6], o[7]);
    else std::printf(" -\n");
  }
  cudaFree(d_in);
  cudaFree(d_out);
  return 0;
}
