// plans.cu -- circuit schedules other than one launch per gate.
#include "internal.cuh"

namespace qsim {


}  // namespace qsim
