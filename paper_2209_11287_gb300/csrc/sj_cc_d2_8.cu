// CUDA-core distance tiles (sj_join_cc.cuh) instantiated for padded dimensions 2, 4, 8.
#include "sj_join_cc.cuh"

namespace sj {

template int launch_cc_dp<float, 2>(Index*, const JoinParams&);
template int launch_cc_dp<double, 2>(Index*, const JoinParams&);
template int launch_cc_dp<float, 4>(Index*, const JoinParams&);
template int launch_cc_dp<double, 4>(Index*, const JoinParams&);
template int launch_cc_dp<float, 8>(Index*, const JoinParams&);
template int launch_cc_dp<double, 8>(Index*, const JoinParams&);

}  // namespace sj
