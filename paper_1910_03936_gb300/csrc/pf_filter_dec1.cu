#define PF_DEC 1
#include "pf_filter_inst.cuh"
