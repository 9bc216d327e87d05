// Force kernels for NGLL = 6 (see sem_forces.cuh).
#define SEM_NGLL 6
#include "sem_forces.cuh"
