// FP64 sweeps on FP64 state (the plain FP64 form).
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(double, double, double, JQ_LINEAR, EPI_STORE)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_ACC_SET)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_ACC_ADD)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_HEAT_FINAL)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_WAVE_FINAL)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_HJ_X)
MOLT_INST(double, double, double, JQ_LINEAR, EPI_HJ_Y)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_STORE)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_HJ_X)
MOLT_INST(double, double, double, JQ_WENOZ, EPI_HJ_Y)
}  // namespace molt
