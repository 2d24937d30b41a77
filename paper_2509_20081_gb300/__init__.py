"""GB300 (sm_103a) DB-TSDF scan integration and map export.

The compute path is libdbtsdf.so (CUDA kernels behind the C ABI of
include/dbtsdf.h); ``dbtsdf`` is its thin ctypes binding.
"""
from . import build  # noqa: F401
from .dbtsdf import (  # noqa: F401
    Batch, DBT_BINS_AZEL, DBT_BINS_OCTA, DbtError, Grid, Kernels, Workspace, dbt_bin_directions,
    dbt_get_scan_stats, dbt_grid_init, dbt_grid_layout, dbt_integrate_scan,
    dbt_integrate_scan_ex, dbt_integrate_scan_host, dbt_integrate_scan_noalloc, dbt_mesh_extract,
    dbt_mesh_centroids, dbt_nn_distances, dbt_pose_ramp, dbt_quality_metrics,
    dbt_mesh_scratch_size, dbt_mesh_table, dbt_read_distance, dbt_read_voxels, dbt_scan_contacts, dbt_sdf_field,
    dbt_sync, dbt_tables_host, dbt_version, lib, make_params)
