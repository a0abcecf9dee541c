"""GB300-native two-level Strang splitting for the spatial fractional
Allen-Cahn equation (arXiv 2209.08437): a CUDA C-ABI library (libsfac) and
its thin Python binding."""
from .sfac import (SFAC_FP32, SFAC_FP64, Batch, Plan, Server, SfacError, SfacParams, load, make_params,  # noqa: F401
                   sfac_axis_pass, sfac_diagnostics, sfac_plan_info, sfac_plan_kernel, sfac_plan_check, sfac_plan_set_wait_limit,
                   SFAC_KERNEL_CTA, SFAC_KERNEL_WARP, SFAC_KERNEL_STAGED, sfac_last_error, sfac_plan_create, sfac_plan_destroy, sfac_plan_tables,
                   sfac_solve, sfac_step, sfac_step_host, sfac_version, sfac_batch_create,
                   sfac_batch_destroy, sfac_batch_prepare, sfac_batch_launch, sfac_batch_wait,
                   sfac_batch_step, sfac_batch_autotune, sfac_batch_set_config, sfac_batch_get_config,
                   sfac_batch_num_configs, sfac_batch_set_wait_limit, sfac_batch_launch_noalloc,
                   sfac_server_create,
                   sfac_server_destroy, sfac_server_request_bytes, sfac_server_admit, sfac_server_round,
                   sfac_server_wait, sfac_server_fetch, sfac_server_info, sfac_server_set_wait_limit,
                   sfac_probe_fma, sfac_probe_jq, sfac_plan_step_kernel, SFAC_STEP_PASSES, SFAC_STEP_WHOLE,
                   sfac_plan_host_route, SFAC_HOST_COPY, SFAC_HOST_MAPPED, SFAC_HOST_MAPPED_IN)
from .serving import serve  # noqa: F401
