// NTT schedules of ring degree 2^12 (see ntt_part.cuh).
#define NTT_LOGN 12
#include "ntt_part.cuh"
