"""GB300-native near-wall refinement of a forest-of-octrees grid around a triangle (segment) mesh.

Data-parallel hot path of Jaber, Essel & Sullivan (2025), "Towards a GPU-native
adaptive mesh refinement scheme for the Lattice Boltzmann Method in complex
geometries": import -> spatial binning -> near-wall refinement with adjacent-face
lists and lattice wall links.  The compute runs in hand-written sm_103a CUDA
kernels behind the C ABI of ``include/amrgeom.h``; this package is its binding.
"""
from .binding import (  # noqa: F401
    AMR_FACE_PASS_AUTO,
    AMR_FACE_PASS_OFF,
    AMR_FACE_PASS_ON,
    AMR_PRED_BOX,
    AMR_PRED_POINT,
    AMR_SEARCH_OWN_BIN,
    AMR_SEARCH_QUERY_BOX,
    EXPORTED,
    AmrError,
    AmrBatch,
    AmrGeom,
    amr_autotune,
    amr_bin_faces,
    amr_bin_faces_sampled,
    amr_bin_faces_static,
    amr_create,
    amr_destroy,
    amr_geom_load,
    amr_launch_count,
    amr_q_backward,
    amr_refine_near_wall,
    amr_set_stream,
    amr_sync,
    amr_timing_enable,
    amr_timing_get,
    amr_timing_reset,
    lib,
    q_links,
)
