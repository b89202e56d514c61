"""The 3D octree code of libfc runs on the host (Morton keys, hash index,
regrid with 2:1 balance over 26 directions, neighbour tables); checked here
without a GPU: random forests and random refine / coarsen flags, the
library's regrid against the 3D oracle's (bit for bit), every neighbour-table
entry against the forest, and the tile / record slots the kernels need."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.fco3 import INIT_GAUSS, Oracle3, Oracle3Params
from paper_1308_1472_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = _build.build()
    exe = str(tmp_path_factory.mktemp("fc3host") / "fc3_host_check")
    # host code is what runs; device code only as PTX to keep the compile short
    cmd = [nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=compute_103a", "-I",
           os.path.join(os.path.dirname(HERE), "include"), os.path.join(HERE, "fc3_host_check.cu"), "-o", exe,
           "-L", os.path.dirname(lib), "-lfc", "-Xlinker", "-rpath=" + os.path.dirname(lib)]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_host_regrid_and_tables_against_oracle(checker, tmp_path, seed):
    rng = np.random.default_rng(seed)
    lmin, lmax = 1, 4
    o = Oracle3(Oracle3Params(m=4, min_level=lmin, max_level=lmax))
    o.init(INIT_GAUSS, [0.2, 1.0, 0.3, 0.6, 0.45, 0.2])
    for r in range(3):
        lv, x, y, z = o.leaves()
        flags = rng.choice(np.array([-1, 0, 1], np.int8), size=o.n, p=[0.35, 0.4, 0.25])
        inp, out = tmp_path / f"in{r}.txt", tmp_path / f"out{r}.txt"
        with open(inp, "w") as fh:
            fh.write(f"{o.n} {lmin} {lmax}\n")
            for k in range(o.n):
                fh.write(f"{lv[k]} {x[k]} {y[k]} {z[k]} {flags[k]}\n")
        res = subprocess.run([checker, str(inp), str(out)], capture_output=True, text=True)
        assert res.returncode == 0 and res.stdout.startswith("ok"), res.stdout + res.stderr
        o.regrid(flags)
        got = np.loadtxt(out, dtype=np.int64, ndmin=2)
        ref = np.stack([a.astype(np.int64) for a in o.leaves()], axis=1)
        assert np.array_equal(got, ref), r
