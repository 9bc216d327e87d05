// Force kernels for NGLL = 10 (see sem_forces.cuh).
#define SEM_NGLL 10
#include "sem_forces.cuh"
