// Kernels of the 1-D configuration with 1 Gauss point(s) per face in double.
#include "kfns_impl.cuh"
namespace cgks {
Kfns kfns_1_1_d(bool one) { return make_kfns<1, 1, double>(one); }
}
