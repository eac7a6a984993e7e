// CUDA-core distance tiles (sj_join_cc.cuh) instantiated for padded dimension 32.
#include "sj_join_cc.cuh"

namespace sj {

template int launch_cc_dp<float, 32>(Index*, const JoinParams&);
template int launch_cc_dp<double, 32>(Index*, const JoinParams&);

}  // namespace sj
