"""GB300-native two-level Strang splitting for the spatial fractional
Allen-Cahn equation (arXiv 2209.08437): a CUDA C-ABI library (libsfac) and
its thin Python binding."""
from .sfac import (SFAC_FP32, SFAC_FP64, Plan, SfacError, SfacParams, load, make_params,  # noqa: F401
                   sfac_axis_pass, sfac_last_error, sfac_plan_create, sfac_plan_destroy, sfac_plan_tables,
                   sfac_solve, sfac_step, sfac_step_host, sfac_version)
