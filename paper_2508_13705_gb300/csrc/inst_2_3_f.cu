// Kernels of the 2-D configuration with 3 Gauss point(s) per face in float.
#include "kfns_impl.cuh"
namespace cgks {
Kfns kfns_2_3_f(bool one) { return make_kfns<2, 3, float>(one); }
}
