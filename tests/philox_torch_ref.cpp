// Test helper: prints Philox4x32-10 blocks computed by PyTorch's ATen
// philox_engine (an implementation independent of this repository's oracle
// and CUDA code).  Reads lines "seed subsequence offset" (decimal u64) from
// stdin and prints the four 32-bit words of that counter block in hex.
// philox_engine(seed, subsequence, offset) keys the cipher with (seed lo,
// seed hi) and sets the counter to (offset lo, offset hi, subseq lo, subseq hi).
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>

int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%08x %08x %08x %08x\n", a, b, c, d);
  }
  return 0;
}
