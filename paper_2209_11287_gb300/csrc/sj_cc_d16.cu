// CUDA-core distance tiles (sj_join_cc.cuh) instantiated for padded dimension 16.
#include "sj_join_cc.cuh"

namespace sj {

template int launch_cc_dp<float, 16>(Index*, const JoinParams&);
template int launch_cc_dp<double, 16>(Index*, const JoinParams&);

}  // namespace sj
