// CUDA-core distance tiles (sj_join_cc.cuh) instantiated for padded dimension 128.
#include "sj_join_cc.cuh"

namespace sj {

template int launch_cc_dp<float, 128>(Index*, const JoinParams&);
template int launch_cc_dp<double, 128>(Index*, const JoinParams&);

}  // namespace sj
