// Kernels of the 2-D configuration with 4 Gauss point(s) per face in float.
#include "kfns_impl.cuh"
namespace cgks {
Kfns kfns_2_4_f(bool one) { return make_kfns<2, 4, float>(one); }
}
