// FP32 compute, FP32 shifted storage of all populations (bulk kernels of two nodes per thread).
#define KTF float
#define KTG float
#define KR float
#define KNAME launchers_f32_n2
#define KPART 2
#include "kernels_impl.cuh"
