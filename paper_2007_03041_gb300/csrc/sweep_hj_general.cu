// Hamilton-Jacobi passes for every Hamiltonian, source terms and speed-only
// passes (FP32 and FP64), compiled apart from the |grad u|^2/2 kernels.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(float, float, float, JQ_LINEAR, EPI_HJ_XG)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_HJ_YG)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_HJ_XG)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_HJ_YG)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_HJ_XG)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_HJ_YG)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_HJ_XG)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_HJ_YG)
}  // namespace molt
