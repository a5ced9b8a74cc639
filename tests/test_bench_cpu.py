"""bench.py on the CPU: the reference arm (the oracle timed on the host cores)
runs end to end and prints the contract's JSON line, and no function of the
script uses a name that is defined nowhere in it."""
import ast
import builtins
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
         "--warmup", "1", "--cpu-seconds", "0.2"],
        cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["workload"] == "sbbf_4194304blk_100M_ins_1G_lookup"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the same config dict as our arm emits for the default workload
    sys.path.insert(0, ROOT)
    import bench
    from paper_2101_01719_gb300 import workloads as wl
    assert line["config"] == bench.workload_config(wl.C2, 1)


def _stored_names(node):
    names = set()
    for n in ast.walk(node):
        if isinstance(n, (ast.Import, ast.ImportFrom)):
            names.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, ast.arg):
            names.add(n.arg)
    return names


def test_bench_uses_no_undefined_names():
    """Each top-level function may use builtins, module-level names and the
    names it (or a function nested in it) binds -- not a local of another
    function."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module = set(dir(builtins)) | {"__file__", "__name__"}
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            module.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            module.add(node.name)
        elif isinstance(node, (ast.Assign, ast.AnnAssign, ast.AugAssign)):
            module |= _stored_names(node)
    missing = {}
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            scope = module | _stored_names(node)
            used = {n.id for n in ast.walk(node)
                    if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
            if used - scope:
                missing[node.name] = sorted(used - scope)
    assert not missing, missing


def test_step_kernel_counts():
    """gpu_launches: a step launches the clear, one kernel per unpartitioned
    batch, three per 2^34-key piece of a partitioned insert batch, four per
    2^31-key piece of a partitioned lookup and one per region pass of an
    insert of hashes or a lookup of hashes or fixed-width keys, plus one
    hashing kernel per partitioned batch of raw keys."""
    sys.path.insert(0, ROOT)
    import bench

    class FakeFilter:
        def __init__(self, ins, look, passes=1, ins_passes=1):
            self.ins, self.look, self.passes, self.ins_passes = ins, look, passes, ins_passes

        def partition_applies(self, n, lookup=False):
            return self.look if lookup else self.ins

        def region_passes(self, n, lookup=True):
            return self.passes if lookup else self.ins_passes

    assert bench.step_kernels(FakeFilter(False, False), [(0, 10)], 100, False) == 3
    assert bench.step_kernels(FakeFilter(False, False), [(0, 10), (10, 5)], 100, True) == 4
    assert bench.step_kernels(FakeFilter(True, True), [(0, 10), (10, 5)], 100, False) == 1 + 6 + 4
    assert bench.step_kernels(FakeFilter(True, False), [(0, 10)], 100, True) == 1 + 4 + 1
    assert bench.step_kernels(FakeFilter(False, True), [(0, 10)], 2**31 + 1, True) == 1 + 1 + 8 + 1
    assert bench.step_kernels(FakeFilter(True, False), [(0, 2**34 + 1)], 1, False) == 1 + 6 + 1
    # a lookup by region passes: one launch per pass (hash lookups only)
    assert bench.step_kernels(FakeFilter(True, False, 2), [(0, 10)], 100, False) == 1 + 3 + 2
    assert bench.step_kernels(FakeFilter(False, False, 3), [(0, 10)], 100, True) == 1 + 1 + 3
    assert bench.step_kernels(FakeFilter(True, False, 2, 2), [(0, 10), (10, 5)], 100,
                              False) == 1 + 2 + 2 + 2
