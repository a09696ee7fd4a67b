// Kernels of the 2-D configuration with 4 Gauss point(s) per face in double.
#include "kfns_impl.cuh"
namespace cgks {
Kfns kfns_2_4_d(bool one) { return make_kfns<2, 4, double>(one); }
}
