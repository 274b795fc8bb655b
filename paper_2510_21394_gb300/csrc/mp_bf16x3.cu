// placeholder: replaced by the tcgen05 kernel
#include "common.h"
#include "engine.h"
namespace fcgle {
void bf16x3_prepare(const double*, int, Bf16x3Op&) { throw Unsupported("BF16X3 not built yet"); }
void bf16x3_release(Bf16x3Op&) {}
void mp_bf16x3(const float*, float*, const Bf16x3Op&, size_t, int*, cudaStream_t, long long&) {}
int bf16x3_num_sms() { return 0; }
}
