"""Host-side checks that need no GPU: the C ABI library loads and exports every entry point the
header declares, the binding refuses to run without it, option marshalling, and the
independent-replica aggregation of the benchmark over two gloo ranks."""
import ctypes
import os
import re
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tuckersgmres.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(tk_\w+)\s*\(", txt, flags=re.M))


def test_header_declares_the_exported_names():
    from paper_2608_11091_b300 import _lib as L
    assert _declared() == set(L.EXPORTS)


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2608_11091_b300 import _lib as L
    assert os.path.exists(L.LIB_PATH), "build the library first: python -m paper_2608_11091_b300.build"
    lib = ctypes.CDLL(L.LIB_PATH)
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_missing_library_fails_loudly(tmp_path):
    from paper_2608_11091_b300 import _lib as L
    with pytest.raises(ImportError):
        L.load(str(tmp_path / "absent.so"))


def test_options_marshalling():
    import workloads as W
    from paper_2608_11091_b300 import _lib as L
    from paper_2608_11091_b300.api import Options
    prm = W.SolverParams('rhosvd', 24, 96, 7, 33, 2e-7, eta=0.4, ktrunc=3, round_tol=1e-11, seed=9)
    c = Options.from_params(prm, precision="mixed", transpose=True).c()
    assert (c.variant, c.rank_cap, c.sketch_s, c.oversample_p, c.ktrunc, c.maxit) == \
        (L.TK_RHOSVD_SGMRES, 24, 96, 7, 3, 33)
    assert (c.tol, c.eta, c.round_tol, c.seed) == (2e-7, 0.4, 1e-11, 9)
    assert c.precision == L.TK_MIXED and c.transpose == 1
    assert Options(variant="mln").c().variant == L.TK_MLN_SGMRES


def test_fortran_layout_helpers():
    import numpy as np
    from paper_2608_11091_b300.api import fortran_empty, is_fortran, to_fortran
    a = np.arange(24.0).reshape(2, 3, 4)
    t = to_fortran(a, "cpu")
    assert is_fortran(t) and np.array_equal(t.numpy(), a)
    assert is_fortran(fortran_empty((5, 6), "cpu"))
    assert not is_fortran(to_fortran(a, "cpu").permute(1, 0, 2))


def _replica_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        # rank r timed 1 + r seconds for 10 (r + 1) iterations
        t, units = bench.aggregate_over_ranks(1.0 + rank, 10.0 * (rank + 1), "cpu")
        wl = W.workload("poisson3d_n32", seed=rank)
        q.put((rank, t, units, float(wl.b.core.ravel()[0])))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, units, _ in out:
        assert t == 2.0 and units == 30.0   # max time over ranks, total iterations of all ranks
    assert out[0][3] != out[1][3]           # each replica solves its own seeded right-hand side


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_over_ranks(1.5, 7, "cpu") == (1.5, 7.0)


def _bench(args, env_extra=None, timeout=300):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=timeout)
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    return p.returncode, [json.loads(ln) for ln in lines]


def test_reference_arm_json_contract():
    """bench.py --impl reference: the oracle timed on the host cores, one JSON line with the
    contract's keys (the reference arm of the benchmark, no GPU involved)."""
    rc, lines = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "poisson3d_smooth_n64"])
    assert rc == 0 and len(lines) == 1
    d = lines[0]
    for key in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["config"]["workload"] == "poisson3d_smooth_n64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    """Under torchrun only rank 0 runs and prints the reference line; the others exit 0 silently."""
    rc, lines = _bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert rc == 0 and lines == []


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has, in the C header compiled by gcc, the same size and
    the same field offsets as its ctypes definition: a field added, dropped, retyped or moved on
    one side only would otherwise corrupt every call silently."""
    import shutil
    import subprocess
    from paper_2608_11091_b300 import _lib as L
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {name: getattr(L, name) for name in ["tk_tucker", "tk_modemat", "tk_operator", "tk_opts", "tk_report",
                                                         "tk_solve_job"]}
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "tuckersgmres.h"', 'int main(void) {']
    for name, cls in structs.items():
        src.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            src.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    src.append('  return 0;\n}')
    c_file, exe = tmp_path / "layout.c", tmp_path / "layout"
    c_file.write_text("\n".join(src) + "\n")
    subprocess.run([gcc, "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(c_file), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
