"""Host checks of the measurement bookkeeping: the algorithmic bytes that
bench.py and dm_bench.py charge per operation (each amplitude an operation
touches read and written once), and the mapping of ncu launch records onto the
bench's kernel families in profile_ops (the DRAM traffic record).  CPU only."""

import csv
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2311_01512_gb300 import dm_bench, profile_ops  # noqa: E402

PASS30 = 2 * 16 * (1 << 30)


def test_statevector_op_bytes():
    u = {"op": "unitary", "ctrls": [], "targs": [3]}
    assert bench.op_bytes(u, 30, 16) == PASS30
    assert bench.op_bytes(dict(u, ctrls=[0, 1]), 30, 16) == PASS30 // 4
    assert bench.op_bytes({"op": "diagonal", "targs": [1, 2]}, 30, 16) == PASS30
    assert bench.op_bytes({"op": "gadget", "targs": [1], "paulis": [1]}, 30, 16) == PASS30
    assert bench.op_family(dict(u, targs=[3, 9])) == "k_dense<2>"
    assert bench.op_family({"op": "gadget", "targs": [1, 2], "paulis": [3, 3]}) == "k_phase"


def test_density_matrix_op_bytes():
    """One pass over the 2N-qubit Choi vector for uncontrolled one- and
    two-qubit unitaries (one pass of conj(U) (x) U), two passes for the others
    (U, then U* on t + N), halved per control; dephasing touches half (one
    qubit) or three quarters (two qubits) of the amplitudes."""
    nq = 15
    full = 32 * (1 << (2 * nq))
    u = {"op": "unitary", "ctrls": [], "targs": [3]}
    assert dm_bench.op_bytes(u, nq) == full
    assert dm_bench.op_bytes(dict(u, targs=[3, 7]), nq) == full
    assert dm_bench.op_bytes(dict(u, targs=[3, 7, 9]), nq) == 2 * full
    assert dm_bench.op_bytes(dict(u, ctrls=[1]), nq) == full
    assert dm_bench.op_bytes(dict(u, ctrls=[1, 2], targs=[3, 7]), nq) == full // 2
    assert dm_bench.op_bytes({"op": "dephasing", "targs": [1]}, nq) == full // 2
    assert dm_bench.op_bytes({"op": "dephasing2", "targs": [1, 2]}, nq) == full * 3 // 4
    assert dm_bench.op_bytes({"op": "kraus", "targs": [1, 2]}, nq) == full


def write_ncu_csv(path, launches):
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
                    "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit",
                    "Metric Value"])
        for i, (name, rd, wr) in enumerate(launches):
            for metric, val in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr),
                                ("gpu__time_duration.sum", 1000)):
                w.writerow([str(i), "1", "python3", "h", name, "1", "13", "(256, 1, 1)", "(38912, 1, 1)", "0",
                            "10.3", "Command line profiler metrics", metric, "byte", "{:,}".format(rd if metric
                            == "dram__bytes_read.sum" else wr if metric == "dram__bytes_write.sum" else 1000)])


def test_traffic_record_family_mapping(tmp_path):
    """Launch records named as ncu prints them, one capture per kernel as the
    profiling sequence makes them, land on the bench's families, scaled from
    28 to 30 qubits (x4)."""
    caps = {
        "g1": [("void k_gate1_fx<1>(double2 *, Gate1FxParams)", 100, 1)],
        "g2": [("void k_gate2_fx<1>(double2 *, Gate2FxParams)", 200, 2)],
        "ws": [("void k_dense_ozaki_ws<3, 8>(double2 *, TcParams)", 300, 3),
               ("void k_dense_ozaki_ws<4, 8>(double2 *, TcParams)", 400, 4)],
        "oz5": [("void k_dense_ozaki<5, 512, 1, 1, 8>(double2 *, TcParams)", 500, 5)],
        "tc": [("void k_dense_tc<5, 256, 1, 2>(float2 *, TcParams)", 600, 6)],
        "diag": [("void k_diag_fx<3>(double2 *, DiagFxParams)", 700, 7)],
        "gad": [("k_gadget_fx(double2 *, GadgetFxParams)", 800, 8)],
        "ph": [("k_phase_fx(double2 *, GadgetFxParams)", 900, 9)],
    }
    paths = []
    for key, launches in caps.items():
        p = tmp_path / (key + ".csv")
        write_ncu_csv(p, launches)
        paths.append(str(p))
    out = tmp_path / "traffic.json"
    profile_ops.summarize_traffic(paths, 28, 30, str(out))
    fam = json.load(open(out))["families"]
    assert fam == {"k_gate1": 404.0, "k_dense<2>": 808.0, "k_dense<3>": 1212.0, "k_dense<4>": 1616.0,
                   "k_dense<5>": 2020.0, "c64 k_dense<5>": 2424.0, "k_diag": 2828.0, "k_gadget": 3232.0,
                   "k_phase": 3636.0}
