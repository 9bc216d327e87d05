// Force kernels for NGLL = 9 (see sem_forces.cuh).
#define SEM_NGLL 9
#include "sem_forces.cuh"
