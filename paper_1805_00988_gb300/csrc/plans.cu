// plans.cu -- circuit schedules other than one launch per gate.
#include "internal.cuh"

namespace qsim {

int apply_circuit_fused(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o)
{
    (void)s; (void)gates; (void)n_gates; (void)o;
    return fail(SIM_EUNSUPPORTED, "fused plan not built yet");
}

}  // namespace qsim
