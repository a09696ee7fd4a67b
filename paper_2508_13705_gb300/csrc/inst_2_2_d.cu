// Kernels of the 2-D configuration with 2 Gauss point(s) per face in double.
#include "kfns_impl.cuh"
namespace cgks {
Kfns kfns_2_2_d(bool one) { return make_kfns<2, 2, double>(one); }
}
