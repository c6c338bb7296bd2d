"""Host-side checks of the benchmark's bookkeeping: every timing site the library records
maps to a kernel the library defines (so the per-kernel table and the roofline see every
launch), the grouping of sites into kernels, and the configuration both arms report."""
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
    sites = {"krylov_multi_dot": (139, 20.0, 1e9, 4e9), "krylov_finalize_dot": (5, 1.0, 1e8, 2e8),
             "krylov_basis_dot": (139, 30.0, 1e9, 2e9),
             "amg_gs_pre_l1": (417, 2.0, 1e8, 0.0), "amg_gs_post_l3": (1390, 5.0, 2e8, 0.0),
             "precond_graph": (139, 200.0, 5e9, 0.0), "setup:galerkin": (1, 30.0, 0.0, 0.0)}
    out = bench.kernels_from_sites(sites)
    assert out["multi_dot1_kernel"] == [144, 21.0, 1.1e9, 4.2e9]
    assert out["ell_gs_colour_kernel"] == [1807, 7.0, 3e8, 0.0]
    assert "precond_graph" not in out and len(out) == 2


def test_roofline_picks_the_binding_roof():
    # 1 GB and 0.25 TFLOP in 1 ms: 1 TB/s of 6.7 TB/s HBM, but 250 TFLOP/s-equivalent work
    # at the FP64 rate: the ALU binds (its time at peak is the longer)
    r = bench.roofline_of("k", [10, 10.0, 1e10, 2.5e12 * 1e-3 * 10], 6763.3, "measured", 152,
                          2070.0, 1.25e12, 100.0, 1)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["peak"] - 152 * 2 * 2 * 2070e6 / 1e12) < 1e-3
    r = bench.roofline_of("k", [10, 10.0, 1e10, 0.0], 6763.3, "measured", 152, 2070.0, 1.25e12,
                          100.0, 1)
    assert r["bound"] == "hbm" and r["achieved"] == 1000.0


def test_static_config_is_shared_by_both_arms():
    import argparse
    from synthetic import grid_spe10
    args = argparse.Namespace(nx=6, ny=5, nz=4, mu=180, precision="fp64", colouring="alg41",
                              smoother="pgs_mc", wells="rows")
    a = grid_spe10(nx=6, ny=5, nz=4)
    c = bench.static_config(args, a)
    assert c["cells"] == 120 and c["block_rows"] == 124 and c["nnzb"] == a.nnzb
    assert "R_ij + 3 I" in c["workload"] and "rebalanced" in c["workload"]


def _bench(args, env=None):
    import json
    import os
    import subprocess
    import sys
    e = dict(os.environ, **(env or {}))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       env=e, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_the_contract_line_on_rank_0_only():
    """The reference arm times the oracle on the host cores: one JSON line on rank 0 with the
    base contract's keys, a cpu_baseline of kind oracle and an e2e without host copies; the
    other ranks print nothing and exit 0."""
    args = ["--impl", "reference", "--nx", "6", "--ny", "5", "--nz", "4", "--steps", "2",
            "--warmup", "1"]
    (line,) = _bench(args)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "solves/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["cells"] == 120
    assert _bench(args, env={"RANK": "1", "WORLD_SIZE": "2"}) == []
