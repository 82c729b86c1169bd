// Draws of C++ standard-library engines that coincide with special cases of
// the paper's generators.  The engines are specified by ISO C++ [rand.eng.lcong],
// [rand.eng.mers], [rand.eng.sub], [rand.adapt.disc]; the library's
// implementation is independent of the oracle under test.
//   usage: stdlib_engines <engine> <seed> <n>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

template <class E>
static void dump(E e, unsigned long long n) {
  for (unsigned long long i = 0; i < n; i++) std::printf("%llu\n", (unsigned long long)e());
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const char* name = argv[1];
  unsigned long long seed = std::strtoull(argv[2], nullptr, 10);
  unsigned long long n = std::strtoull(argv[3], nullptr, 10);
  typedef std::linear_congruential_engine<std::uint_fast32_t, 40014u, 0u, 2147483563u> lcg1;
  typedef std::linear_congruential_engine<std::uint_fast32_t, 40692u, 0u, 2147483399u> lcg2;
  if (!std::strcmp(name, "minstd_rand0")) dump(std::minstd_rand0(seed), n);
  else if (!std::strcmp(name, "mt19937")) dump(std::mt19937(seed), n);
  else if (!std::strcmp(name, "ranlux24_base")) dump(std::ranlux24_base(seed), n);
  else if (!std::strcmp(name, "ranlux_p48")) dump(std::discard_block_engine<std::ranlux24_base, 48, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p97")) dump(std::discard_block_engine<std::ranlux24_base, 97, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p223")) dump(std::discard_block_engine<std::ranlux24_base, 223, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p389")) dump(std::discard_block_engine<std::ranlux24_base, 389, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p120")) dump(std::discard_block_engine<std::ranlux24_base, 120, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p240")) dump(std::discard_block_engine<std::ranlux24_base, 240, 24>(seed), n);
  else if (!std::strcmp(name, "ranlux_p408")) dump(std::discard_block_engine<std::ranlux24_base, 408, 24>(seed), n);
  else if (!std::strcmp(name, "lcg40014")) dump(lcg1(seed), n);
  else if (!std::strcmp(name, "lcg40692")) dump(lcg2(seed), n);
  else return 3;
  return 0;
}
