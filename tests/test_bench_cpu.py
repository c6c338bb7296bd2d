"""Host-side checks of the benchmark's bookkeeping: every timing site the library records
maps to a kernel the library defines (so the per-kernel table and the roofline see every
launch), the grouping of sites into kernels, and the FP64 ceiling arithmetic."""
import glob
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2208_08594_gb300", "csrc")


def _sources():
    return "\n".join(open(f).read() for f in glob.glob(os.path.join(CSRC, "*.cu")))


def _kernels(src):
    return set(re.findall(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?(\w+)\s*\(", src))


def _sites(src):
    exact = set(re.findall(r'Probe\s+\w+\("([A-Za-z0-9_:]+)"', src))
    prefixes = set(re.findall(r'level_site\("([a-z_]+)"', src))
    prefixes |= set(re.findall(r'"(amg_gs_[a-z_]+_l)"', src))
    return exact, prefixes


def test_every_timed_site_maps_to_a_defined_kernel():
    src = _sources()
    kernels = _kernels(src)
    exact, prefixes = _sites(src)
    assert "krylov_multi_dot" in exact and "amg_gs_pre_l" in prefixes
    # sites that time more than one kernel or host work are not kernel rows
    grouped = {"precond_graph"} | {s for s in exact if s.startswith("setup:")}
    for site in sorted(exact - grouped):
        k = bench.SITE_KERNELS.get(site)
        assert k is not None, site
        assert k in kernels, (site, k)
    for p in sorted(prefixes):
        k = bench.SITE_PREFIX_KERNELS.get(p)
        assert k is not None, p
        assert k in kernels, (p, k)


def test_kernels_from_sites_groups_by_kernel():
    sites = {"krylov_multi_dot": (139, 20.0, 1e9), "krylov_reorth_dot": (139, 22.0, 1e9),
             "amg_gs_pre_l1": (417, 2.0, 1e8), "amg_gs_post_l3": (1390, 5.0, 2e8),
             "precond_graph": (139, 200.0, 5e9), "setup:galerkin": (1, 30.0, 0.0)}
    out = bench.kernels_from_sites(sites)
    assert out["multi_dot_kernel"] == [278, 42.0, 2e9]
    assert out["ell_gs_colour_kernel"] == [1807, 7.0, 3e8]
    assert "precond_graph" not in out and len(out) == 2


def test_fp64_fma_ceiling():
    # one FMA per 8-byte value at 1.19 TFLOP/s (two flops per FMA)
    assert abs(bench.FP64_FMA_CEILING_GBPS - 4760.0) < 1e-6
