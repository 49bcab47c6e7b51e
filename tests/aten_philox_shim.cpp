// Third-party Philox4x32-10 (ATen's philox_engine) exposed as a C function, so
// the oracle's own generator can be checked against an implementation it
// shares no code with.  Built by tests/thirdparty.py into a temp directory.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
extern "C" void aten_philox_words(uint64_t seed, uint64_t subsequence, uint64_t offset, uint32_t* out4) {
  at::philox_engine e(seed, subsequence, 0);
  e.set_offset(offset);
  for (int i = 0; i < 4; ++i) out4[i] = e();
}
