// FP64 storage and compute.
#define KTF double
#define KTG double
#define KR double
#define KNAME launchers_f64
#define KPART 1
#include "kernels_impl.cuh"
