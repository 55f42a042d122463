// k_dop853_q3.cu -- fixed-step DOP853 integrate kernels of the coupled quartic
// oscillator (3 DOF, up to 6 deviation vectors), compiled apart from the 2-DOF
// systems' (k_dop853.cu) so that the two build in parallel.
#include "k_dop853.cuh"
#include "k_dop853_fixed.cuh"

namespace chs {

cudaError_t launch_integrate_dp_q3(int k, bool ld, const StepArgs& a, const SysPar& sp, const EnsPtrs& e,
                                   const OrbitList* ol, cudaStream_t st)
{
    return fixed_sys<SysQuartic3>(k, ld, a, sp, e, ol, st);
}

}  // namespace chs
