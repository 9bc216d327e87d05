// Force kernels for NGLL = 3 (see sem_forces.cuh).
#define SEM_NGLL 3
#include "sem_forces.cuh"
