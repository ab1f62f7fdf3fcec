"""Host logic of bench.py (no GPU): the algorithmic byte counts behind the
roofline fractions, and the DRAM-traffic lookup that ties the committed ncu
figures to the step-kernel source."""
import hashlib
import os

import bench


def test_algorithmic_bytes_per_step():
    # 201^3, FEM cube 101^3, FP32: 36 B per node, 8 B per FEM-updated node
    # (99^3), and in the adjoint 12 B per free node (97^3)
    fwd, adj = bench.algorithmic_bytes(201, 101, 4)
    assert fwd == 36 * 201 ** 3 + 8 * 99 ** 3 == 300_104_028
    assert adj == fwd + 12 * 97 ** 3 == 311_056_104
    # FP64 doubles every term
    f64, a64 = bench.algorithmic_bytes(201, 101, 8)
    assert (f64, a64) == (2 * fwd, 2 * adj)


def test_traffic_lookup_sums_the_kernels_of_a_step_and_checks_the_source():
    vals = {}
    for line in open(bench.TRAFFIC_FILE):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=", 1)
            vals[k.strip()] = v.split("#", 1)[0].strip()
    src = hashlib.sha256(open(bench.STEP_SRC, "rb").read()).hexdigest()[:16]
    keys = ("batched_adjoint_full_dram_bytes", "batched_adjoint_lean_dram_bytes")
    got = bench.traffic_per_launch(*keys)
    if vals["source_sha256_16"] == src:
        assert got == sum(float(vals[k]) for k in keys)
    else:                      # figures taken on another source: not reported
        assert got is None
    assert bench.traffic_per_launch("no_such_kernel") is None
