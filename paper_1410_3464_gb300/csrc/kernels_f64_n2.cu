// FP64 storage and compute (bulk kernels of two nodes per thread).
#define KTF double
#define KTG double
#define KR double
#define KNAME launchers_f64_n2
#define KPART 2
#include "kernels_impl.cuh"
