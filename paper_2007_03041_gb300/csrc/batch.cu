// The batched heat kernel (csrc/batch.cuh) in a translation unit of its own:
// its 512-thread CTAs run two to an SM with no registers to spare, so the
// FP32 <-> FP64 conversions select the hardware conversion in place instead
// of calling it for rare operands.
#define MOLT_CONV_SELECT 1
#define MOLT_BATCH_KERNEL_TU
#include "batch.cuh"
