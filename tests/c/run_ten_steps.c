/* Example of the C ABI: compiled and linked against include/dg.h, libdg.so and
 * the CUDA runtime by tests/test_abi.py (running it needs a GPU). */
#include <cuda_runtime.h>
#include "dg.h"

/* 64^3 cells, k = 3 (b = 20 modes per field), x3 transforms, SSP-RK3, vNR
 * viscosity, Mach-3 OU driving: ten steps of a state held in host memory
 * ([cell][rho, m_x, m_y, m_z][mode], FP32). */
int run_ten_steps(const float* u_host, float* u_out)
{
    const dg_mesh mesh = {{64, 64, 64}, {1.0, 1.0, 1.0}};
    const int order = 3, b = 20;
    const size_t ncell = (size_t)64 * 64 * 64, state = ncell * 4 * b * sizeof(float);
    dg_nu_params nu = {0};
    nu.mode = DG_AV_VNR;
    nu.alpha = 2.0;
    nu.beta = 0.2;
    nu.rho_floor = 1e-3;
    size_t scratch = 0, vhat = 0;
    if (dg_scratch_bytes(&mesh, order, &nu, &scratch) != DG_OK ||
        dg_vhat_bytes(&mesh, order, DG_PREC_X3, &vhat) != DG_OK)
        return DG_EINVAL;
    dg_opts o = {0};
    o.precision = DG_PREC_X3;
    o.rk_stages = 3;
    o.cfl = 0.3;
    cudaStream_t st;
    cudaStreamCreate(&st);
    o.stream = st;
    for (int i = 0; i < 3; ++i) cudaMalloc(&o.u[i], state);
    cudaMalloc(&o.vhat, vhat);  /* cudaMalloc memory is 256-byte aligned */
    cudaMalloc(&o.ahat, ncell * 3 * b * sizeof(float));
    cudaMalloc(&o.scratch, scratch);
    o.scratch_bytes = scratch;

    dg_ctx* ctx = NULL;
    int rc = dg_init(&ctx, &mesh, order, 1.0, &nu, &o);
    const dg_forcing f = {1, 1, 9, 0.5, 3.0, 0, 0.0};  /* on, 1 <= |k|^2 <= 9, zeta, Mach, seed, t_off */
    double t = 0.0, dt = 0.0;
    if (rc == DG_OK) rc = dg_set_state(ctx, u_host, 1);
    if (rc == DG_OK) rc = dg_set_forcing(ctx, &f);
    if (rc == DG_OK) rc = dg_step(ctx, 10, 0.0, &t, &dt);
    if (rc == DG_OK) rc = dg_get_state(ctx, u_out, 1);
    dg_free(ctx);
    for (int i = 0; i < 3; ++i) cudaFree(o.u[i]);
    cudaFree(o.vhat);
    cudaFree(o.ahat);
    cudaFree(o.scratch);
    cudaStreamDestroy(st);
    return rc;
}
