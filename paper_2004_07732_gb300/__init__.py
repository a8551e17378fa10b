"""GB300-native domain-wall multigrid (arXiv:2004.07732) -- Python binding of libdwfmg.so.

All arithmetic runs in the library's sm_103a CUDA kernels behind the C ABI of
include/dwf.h; this package only marshals torch tensors to device pointers.
"""
from ._lib import (  # noqa: F401
    DwfError, Geom, SolveStats, PREC, lib, make_geom, spinor_size, link_size, spinor_dtype,
    links_to, dwf_apply, pv_apply, dwf_pvdag_apply, dwf_pvdag_apply_noalloc, dwf_dot, cgne_solve, bicgstab_solve,
    links_from_angles, gamma5_reflect, link_force, link_grad, dwf_apply_batched, BatchedApply, check_wait_timeout, dwf_apply_host,
    packed_spinor_size, packed_link_size, pack_links, pack_spinor, unpack_spinor, dwf_apply_packed,
    dwf_mobius_apply, dwf_pv_poly_apply,
)
from ._lib import (  # noqa: F401
    MgParams, Multigrid, mg_default_params, mg_setup, mg_solve, mg_destroy, mg_get_prolongator,
    mg_get_null_vectors, mg_get_coarse_links, mg_restrict, mg_prolong, mg_coarse_apply, mg_coarse_apply_multi,
    mg_solve_batched, mg_solve_groups, mg_coarse_tc_form, mg_check_operator,
    LevelParams, mg_default_level_params, mg_add_level, mg_level_get, mg_level_apply, mg_level_restrict,
    mg_level_prolong, mg_level_coarsest_solve, mg_level_ritz_values, mg_level_last_iterations, mg_level_deflation_info,
    mg_transfer_colinearity, mg_transfer_oblique, mg_coarse_solve,
)
from .autograd import DwfSolve, DwfSolveLinks, solve, solve_links  # noqa: F401,E402
