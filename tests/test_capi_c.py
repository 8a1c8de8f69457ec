"""The C ABI called from plain C programs compiled with gcc against include/eat.h and
linked with libeat.so: host-only calls without a GPU (tests/c/abi_host.c), and queries on
device 0 whose rows are compared with the oracle (tests/c/abi_device.c, marked gpu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_1912_00966_gb300")


def test_c_program_uses_the_abi(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    if not os.path.exists(os.path.join(LIBDIR, "libeat.so")):
        pytest.skip("libeat.so not built")
    exe = tmp_path / "abi_host"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", LIBDIR, "-leat",
                    f"-Wl,-rpath,{LIBDIR}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["small", "city"])
def test_c_program_runs_queries_on_the_gpu(tmp_path, which):
    """A plain C program (tests/c/abi_device.c) builds a network on device 0 through the C
    ABI and runs eat_query and eat_query_batch with host buffers; every row it writes
    equals the oracle's."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import oracle
    import synth
    tt = synth.small_grid() if which == "small" else synth.city()
    q = synth.random_queries(tt, 24, 0xCC)
    tfile, qfile, ofile = tmp_path / "tt.bin", tmp_path / "q.bin", tmp_path / "rows.bin"
    with open(tfile, "wb") as f:
        f.write(np.int32(tt.n_stops).tobytes() + np.int64(tt.n_conn).tobytes())
        for a in (tt.u, tt.v, tt.dep, tt.dur):
            f.write(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    with open(qfile, "wb") as f:
        f.write(np.int32(len(q)).tobytes() + q.source.astype(np.int32).tobytes() +
                q.t_s.astype(np.int32).tobytes())
    exe = tmp_path / "abi_device"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_device.c"), "-L", LIBDIR, "-leat",
                    f"-Wl,-rpath,{LIBDIR}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), str(tfile), str(qfile), str(ofile)], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"
    rows = np.fromfile(ofile, dtype=np.int32).reshape(2, len(q), tt.n_stops)
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    assert np.array_equal(rows[0], want)
    assert np.array_equal(rows[1], want)
