// Force kernels for NGLL = 7 (see sem_forces.cuh).
#define SEM_NGLL 7
#include "sem_forces.cuh"
