// sw.cu -- Stillinger-Weber three-body forces (Sec. 3.3.2).
#include "common.cuh"
#include "kernels.cuh"

md_status md_energy_forces_sw(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb, float *d_f,
                              double *d_E, uint32_t *d_status, md_stream_t stream)
{
    (void)s; (void)p; (void)d_r; (void)nb; (void)d_f; (void)d_E; (void)d_status; (void)stream;
    return MD_ERR_INVALID;
}
