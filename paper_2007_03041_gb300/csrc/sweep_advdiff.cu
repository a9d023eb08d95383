// Sweeps of the advection-diffusion step: acc += coef * S (FP64, FP32 and
// mixed forms), compiled apart from the other epilogues.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(double, double, double, JQ_LINEAR, EPI_ACC_AXPY)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_ACC_AXPY)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_ACC_AXPY)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_ACC_AXPY)
MOLT_INST(float, float, double, JQ_LINEAR, EPI_ACC_AXPY)
}  // namespace molt
