"""GB300-native multi-stage preconditioned FGMRES for fully implicit compositional
Jacobians (block-sparse), after Zhao, Zhang, Feng and Shu (2022).

The solver is the C-ABI library ``libmsp.so`` (declared in ``include/msp.h``); this
package holds its CUDA sources (``csrc/``), the in-tree build (``build.py``) and a thin
ctypes binding (``_native``) plus a small convenience wrapper (``Solver``).
"""
from __future__ import annotations

from . import _native
from ._native import (msp_level_tiles, msp_wells_setup_scalar, msp_wells_update_values_scalar,
                      msp_wells_pack_rhs, msp_wells_unpack,MSP_NOT_CONVERGED, MSP_OK, MSP_PREC_MSP, MSP_PREC_N_ONLY, MSP_PREC_NONE,
                      MSP_PREC_P_ONLY, MSP_PREC_R_ONLY, MSP_PRECISION_FP32, MSP_PRECISION_FP64,
                      MSP_COLOURING_ALG41, MSP_COLOURING_JP, MSP_SMOOTHER_PGS_MC,
                      MSP_SMOOTHER_PJAC, MSP_SMOOTHER_PGS_NO,
                      MspError, msp_apply_precond, msp_colour0, msp_config_default, msp_free,
                      msp_level_get, msp_level_info, msp_num_levels, msp_setup, msp_solve,
                      msp_solve_host, msp_spmv, msp_status_string, msp_update_values,
                      msp_update_values_host, msp_stats_enable, msp_stats_reset,
                      msp_stats_launches, msp_stats_get, msp_vertices_grouping_noalloc,
                      NOALLOC_MAX_VERTICES, msp_fma_rate, msp_wells_setup, msp_wells_reduced,
                      msp_wells_update_values, msp_wells_reduce_rhs, msp_wells_recover,
                      msp_wells_free, msp_device_bytes, msp_estimate_device_bytes,
                      msp_server_create, msp_server_submit, msp_server_wait,
                      msp_server_get_stats, msp_server_free, MspRequest, MSP_REQ_NEW_PATTERN,
                      MSP_REQ_RELEASE, MSP_EXEC_RUN, MSP_EXEC_RELEASE, MSP_SERVER_EXEC_FN,
                      msp_set_instances, msp_solve_batch, msp_stage_values_host,
                      msp_update_values_staged)

__all__ = ["msp_level_tiles", "Solver", "Wells", "ScalarWells", "WellEliminatedSolver",
           "msp_wells_setup_scalar", "msp_wells_update_values_scalar", "msp_wells_pack_rhs",
           "msp_wells_unpack", "Server", "BatchSolver",
           "stack_block_diagonal", "msp_set_instances", "msp_solve_batch", "MspError",
           "msp_stage_values_host", "msp_update_values_staged",
           "msp_wells_setup",
           "msp_device_bytes", "msp_estimate_device_bytes", "msp_server_create",
           "msp_server_submit", "msp_server_wait", "msp_server_get_stats", "msp_server_free",
           "MspRequest", "MSP_REQ_NEW_PATTERN", "MSP_REQ_RELEASE", "MSP_EXEC_RUN",
           "MSP_EXEC_RELEASE", "MSP_SERVER_EXEC_FN",
           "msp_wells_reduced", "msp_wells_update_values", "msp_wells_reduce_rhs",
           "msp_wells_recover", "msp_wells_free", "msp_setup", "msp_update_values", "msp_update_values_host",
           "msp_stats_enable", "msp_stats_reset", "msp_stats_launches", "msp_stats_get",
           "msp_vertices_grouping_noalloc", "NOALLOC_MAX_VERTICES", "msp_fma_rate",
           "msp_solve",
           "msp_solve_host", "msp_free", "msp_apply_precond", "msp_spmv", "msp_num_levels",
           "msp_level_info", "msp_level_get", "msp_colour0", "msp_config_default",
           "msp_status_string", "MSP_OK", "MSP_NOT_CONVERGED", "MSP_PREC_MSP", "MSP_PREC_NONE",
           "MSP_PREC_R_ONLY", "MSP_PREC_P_ONLY", "MSP_PREC_N_ONLY", "MSP_PRECISION_FP64",
           "MSP_PRECISION_FP32", "MSP_COLOURING_ALG41", "MSP_COLOURING_JP",
           "MSP_SMOOTHER_PGS_MC", "MSP_SMOOTHER_PJAC", "MSP_SMOOTHER_PGS_NO"]


class Solver:
    """Owns one solver handle for a BSR matrix held in CUDA tensors.

    ``row_ptr``/``col_idx`` int32 and ``values`` float64 (nnzb*b*b, row-major blocks) on
    the current CUDA device; ``config`` keys are the fields of ``msp_config``.
    """

    def __init__(self, nb, b, row_ptr, col_idx, values, stream=None, **config):
        self.nb, self.b = int(nb), int(b)
        self.cfg = msp_config_default(**config)
        self.h = msp_setup(self.cfg, self.nb, self.b, row_ptr, col_idx, values, stream)

    def update_values(self, values, stream=None):
        msp_update_values(self.h, values, stream)

    def update_values_host(self, values, stream=None):
        msp_update_values_host(self.h, values, stream)

    def stage_values_host(self, values, stream=None):
        """Enqueue the copy of the next values (host array) on `stream` and return."""
        msp_stage_values_host(self.h, values, stream)

    def update_values_staged(self, stream=None):
        """Apply the values of the last stage_values_host once their copy has landed."""
        msp_update_values_staged(self.h, stream)

    def solve(self, rhs, x, rel_tol=1e-6, stream=None):
        return msp_solve(self.h, rhs, x, rel_tol, stream)

    def solve_host(self, rhs, x, rel_tol=1e-6, stream=None):
        return msp_solve_host(self.h, rhs, x, rel_tol, stream)

    def apply_precond(self, g, w, stream=None):
        msp_apply_precond(self.h, g, w, stream)

    def spmv(self, x, y, stream=None):
        msp_spmv(self.h, x, y, stream)

    @property
    def num_levels(self):
        return msp_num_levels(self.h)

    def level(self, l):
        return msp_level_get(self.h, l)

    def colour0(self):
        return msp_colour0(self.h, self.nb)

    def close(self):
        if self.h:
            msp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Wells:
    """Schur-complement elimination of the well unknowns (the last ``nw`` block rows) of a
    BSR matrix held in CUDA tensors: ``A_S = A_RR - A_RW A_WW^-1 A_WR`` on the cell rows.
    ``reduced()`` gives zero-copy views of the reduced matrix (valid while this object
    lives)."""

    def __init__(self, nb, b, nw, row_ptr, col_idx, values, stream=None):
        self.nb, self.b, self.nw = int(nb), int(b), int(nw)
        self.W = msp_wells_setup(self.nb, self.b, self.nw, row_ptr, col_idx, values, stream)
        self.nr, self.row_ptr, self.col_idx, self.values = msp_wells_reduced(self.W, self.b)

    def reduced(self):
        return self.row_ptr, self.col_idx, self.values

    def update_values(self, values, stream=None):
        msp_wells_update_values(self.W, values, stream)

    def reduce_rhs(self, g, gs, stream=None):
        msp_wells_reduce_rhs(self.W, g, gs, stream)

    def recover(self, g, xs, x, stream=None):
        msp_wells_recover(self.W, g, xs, x, stream)

    def close(self):
        if self.W:
            self.row_ptr = self.col_idx = self.values = None
            msp_wells_free(self.W)
            self.W = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ScalarWells(Wells):
    """Elimination of wells with one unknown each (bottom-hole pressure): the cell matrix
    A_RR (``nr`` block rows) plus, per well, its perforated cells (``well_ptr``,
    ``well_cells``), ``arw``/``awr`` (b values per perforation) and ``aww`` (one per
    well).  Vectors of ``reduce_rhs``/``recover`` are in the padded layout of ``nr + nw``
    block rows; ``pack_rhs``/``unpack`` convert."""

    def __init__(self, nr, b, nw, row_ptr, col_idx, values, well_ptr, well_cells, arw, awr,
                 aww, stream=None):
        self.nb, self.b, self.nw = int(nr) + int(nw), int(b), int(nw)
        self.W = msp_wells_setup_scalar(int(nr), self.b, self.nw, row_ptr, col_idx, values,
                                        well_ptr, well_cells, arw, awr, aww, stream)
        self.nr, self.row_ptr, self.col_idx, self.values = msp_wells_reduced(self.W, self.b)

    def update_values(self, values, arw=None, awr=None, aww=None, stream=None):
        msp_wells_update_values_scalar(self.W, values, arw, awr, aww, stream)

    def pack_rhs(self, gr, gw, g, stream=None):
        msp_wells_pack_rhs(self.W, gr, gw, g, stream)

    def unpack(self, x, xr, xw, stream=None):
        msp_wells_unpack(self.W, x, xr, xw, stream)


class WellEliminatedSolver:
    """FGMRES + MSP on the reduced system of :class:`Wells`: ``solve`` forms the reduced
    right-hand side, solves on the cell rows and recovers the well unknowns."""

    def __init__(self, nb, b, nw, row_ptr, col_idx, values, stream=None, **config):
        import torch
        self.wells = Wells(nb, b, nw, row_ptr, col_idx, values, stream)
        rp, ci, v = self.wells.reduced()
        self.solver = Solver(self.wells.nr, b, rp, ci, v, stream, **config)
        n = self.wells.nr * b
        self.gs = torch.empty(n, dtype=torch.float64, device=values.device)
        self.xs = torch.empty(n, dtype=torch.float64, device=values.device)

    def update_values(self, values, stream=None):
        self.wells.update_values(values, stream)
        self.solver.update_values(self.wells.values, stream)

    def solve(self, rhs, x, rel_tol=1e-6, stream=None):
        """Solve with the full right-hand side ``rhs`` (nb*b) into ``x`` (nb*b); the
        tolerance applies to the reduced system."""
        self.wells.reduce_rhs(rhs, self.gs, stream)
        info = self.solver.solve(self.gs, self.xs, rel_tol, stream)
        self.wells.recover(rhs, self.xs, x, stream)
        return info

    def close(self):
        self.solver.close()
        self.wells.close()


class Server:
    """Request loop over the solver (``msp_server_*``): solves of many systems, each kept
    resident on the device under its key between requests (the adaptive SETUP reuses its
    preconditioner), run concurrently by ``slots`` workers with one CUDA stream each and
    admitted by a device-memory budget.  Arrays are host numpy arrays; they are kept alive
    here until :meth:`wait` returns their ticket."""

    def __init__(self, slots=4, hbm_budget=150 * 10**9, device=0, exec_fn=None, **config):
        self.cfg = msp_config_default(**config)
        self._exec = exec_fn
        self.S = msp_server_create(slots, int(hbm_budget), self.cfg, device, exec_fn)
        self._keep = {}

    def submit(self, key, nb, b, rhs, x, values=None, row_ptr=None, col_idx=None, nnzb=None,
               rel_tol=1e-6, new_pattern=False, release=False):
        import numpy as np

        def arr(a, dtype, name):
            if a is None:
                return None
            if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
                raise TypeError("%s must be a C-contiguous numpy array of %s" % (name, dtype))
            return a

        rp, ci = arr(row_ptr, np.int32, "row_ptr"), arr(col_idx, np.int32, "col_idx")
        v, g, xx = arr(values, np.float64, "values"), arr(rhs, np.float64, "rhs"), arr(x, np.float64, "x")
        if nnzb is None:
            if ci is None:
                raise ValueError("nnzb is needed when col_idx is not given")
            nnzb = ci.size
        if g.size != nb * b or xx.size != nb * b:
            raise ValueError("rhs and x must have nb*b entries")
        if v is not None and v.size != nnzb * b * b:
            raise ValueError("values must have nnzb*b*b entries")
        req = MspRequest()
        req.key, req.nb, req.b, req.nnzb = int(key), int(nb), int(b), int(nnzb)
        req.h_row_ptr = rp.ctypes.data if rp is not None else None
        req.h_col_idx = ci.ctypes.data if ci is not None else None
        req.h_values = v.ctypes.data if v is not None else None
        req.h_rhs, req.h_x = g.ctypes.data, xx.ctypes.data
        req.rel_tol = float(rel_tol)
        req.flags = (MSP_REQ_NEW_PATTERN if new_pattern else 0) | (MSP_REQ_RELEASE if release else 0)
        t = msp_server_submit(self.S, req)
        self._keep[t] = (rp, ci, v, g, xx)
        return t

    def wait(self, ticket, timeout=-1.0):
        r = msp_server_wait(self.S, ticket, timeout)
        if r is not None:
            self._keep.pop(ticket, None)
        return r

    def stats(self):
        return msp_server_get_stats(self.S)

    def close(self):
        if self.S:
            msp_server_free(self.S)
            self.S = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stack_block_diagonal(mats):
    """Stack BSR matrices with one block size into one block-diagonal BSR matrix (host numpy
    arrays).  ``mats``: objects with ``nb, b, row_ptr, col_idx, values``.  Returns
    (nb, b, row_ptr, col_idx, values (flat), offsets) with offsets[k] the first block row of
    instance k."""
    import numpy as np
    b = int(mats[0].b)
    if any(int(m.b) != b for m in mats):
        raise ValueError("all instances need the same block size")
    offsets = np.zeros(len(mats) + 1, np.int64)
    for k, m in enumerate(mats):
        offsets[k + 1] = offsets[k] + int(m.nb)
    nnz = np.cumsum([0] + [int(m.row_ptr[-1]) for m in mats])
    rp = np.concatenate([np.asarray(m.row_ptr[:-1], np.int64) + nnz[k] for k, m in enumerate(mats)]
                        + [np.array([nnz[-1]])])
    ci = np.concatenate([np.asarray(m.col_idx, np.int64) + offsets[k] for k, m in enumerate(mats)])
    v = np.concatenate([np.asarray(m.values, np.float64).reshape(-1) for m in mats])
    return (int(offsets[-1]), b, rp.astype(np.int32), ci.astype(np.int32), v,
            offsets.astype(np.int32))


class BatchSolver(Solver):
    """A :class:`Solver` over a block-diagonal stack of independent instances (see
    :func:`stack_block_diagonal`): one preconditioner and one launch per kernel serve every
    instance, each instance gets its own FGMRES.  ``offsets``: host sequence of the
    instances' first block rows plus nb."""

    def __init__(self, nb, b, row_ptr, col_idx, values, offsets, stream=None, **config):
        super().__init__(nb, b, row_ptr, col_idx, values, stream, **config)
        self.count = len(offsets) - 1
        msp_set_instances(self.h, offsets)

    def solve_batch(self, rhs, x, rel_tol=1e-6, stream=None):
        return msp_solve_batch(self.h, self.count, rhs, x, rel_tol, stream)
