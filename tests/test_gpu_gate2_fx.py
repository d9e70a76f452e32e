"""Two-target gates in complex128 block fixed point (k_gate2_fx) and the paths
that route to it, against the CPU oracle.

- Statevector gates on two targets, with and without controls, at 26 qubits:
  2^24 quads, more than the grid's threads, so every thread's grid-stride
  loop repeats.
- A one-qubit unitary on a density matrix as one pass of conj(U) (x) U, and a
  one-qubit Kraus map as one pass of its superoperator sum_m conj(K_m) (x) K_m,
  whose constants the library makes on the host (Sec. "Kraus map").
- The tensor-core form of two-target gates, which fused blocks still take
  through qs_apply_dense_block: eight integer slices on the three-target
  kernel with an identity on a free qubit.
"""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def fx_state(qs, nq, density=False, arith=None):
    st = qs.State(nq, density=density, prec=1)
    if arith is not None:
        qs.qs_set_arithmetic(st.handle, arith)
    return st


@pytest.mark.parametrize("targs,ctrls", [([25, 0], []), ([3, 17], []), ([1, 0], []), ([20, 6], [11])])
def test_two_target_whole_state_26_qubits(qs, targs, ctrls):
    nq = 26
    rng = np.random.default_rng(4100 + 7 * targs[0] + targs[1] + len(ctrls))
    psi = wl.random_statevector(nq, rng)
    mat = wl.haar_unitary(4, rng)
    want = orc.apply_ctrl_multi_target(psi, ctrls, targs, mat)
    st = fx_state(qs, nq)
    st.set_amps(psi)
    qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, mat)
    got = st.get_amps()
    st.close()
    scale = float(np.max(np.abs(psi)))
    # per real output: 2^-53 |y| + 2^-54 max|x| max|m| (block fixed point, eight terms)
    assert float(np.max(np.abs(got - want))) <= 2.0 ** -49 * scale


@pytest.mark.parametrize("kind", ["haar", "wide", "zeros"])
def test_two_target_matrix_kinds(qs, kind):
    """A non-unitary matrix whose rows span 1e-8..1e3 (each output row has
    its own exponent), and a state that is zero on most quads."""
    nq = 14
    rng = np.random.default_rng(4200 + len(kind))
    psi = wl.random_statevector(nq, rng)
    mat = wl.haar_unitary(4, rng)
    if kind == "wide":
        mat = mat * 10.0 ** rng.uniform(-8, 3, size=mat.shape)
    if kind == "zeros":
        psi = np.zeros_like(psi)
        psi[rng.choice(psi.size, 7, replace=False)] = rng.standard_normal(7)
    for targs, ctrls in (([5, 9], []), ([13, 2], [0, 7])):
        want = orc.apply_ctrl_multi_target(psi, ctrls, targs, mat)
        st = fx_state(qs, nq)
        st.set_amps(psi)
        qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, mat)
        got = st.get_amps()
        st.close()
        # each row's own scale: |delta y_j| <= 2^-52 (|y_j| + 8 max|x| max_k |m_jk|)
        row_max = np.abs(mat).max(axis=1)
        bound = 2.0 ** -50 * (np.abs(want) + 8 * float(np.max(np.abs(psi))) * row_max.max()) + 1e-300
        assert np.all(np.abs(got - want) <= bound)


def test_density_one_qubit_unitary_and_kraus_13_qubits(qs):
    """13-qubit density matrix (26-qubit Choi vector: the loops repeat): a
    one-qubit unitary on a low and a high qubit, then a two-operator Kraus map,
    each one pass, against the oracle; the result is also compared with the
    two-pass native-FP64 path."""
    nq = 13
    rng = np.random.default_rng(4300)
    pure = [wl.random_statevector(nq, rng) for _ in range(2)]
    rho = 0.7 * orc.densmatr_from_pure(pure[0]) + 0.3 * orc.densmatr_from_pure(pure[1])
    u0, u1 = wl.haar_unitary(2, rng), wl.haar_unitary(2, rng)
    kraus = wl.haar_kraus(1, 2, rng)
    want = orc.densmatr_apply_ctrl_multi_target(rho, [], [0], u0)
    want = orc.densmatr_apply_ctrl_multi_target(want, [], [12], u1)
    want = orc.densmatr_apply_kraus(want, [5], kraus)
    outs = []
    for arith in (None, qs.QS_ARITH_F64):
        st = fx_state(qs, nq, density=True, arith=arith)
        st.set_amps(rho)
        qs.qs_apply_ctrl_multi_target(st.handle, [], [0], u0)
        qs.qs_apply_ctrl_multi_target(st.handle, [], [12], u1)
        qs.qs_apply_kraus(st.handle, [5], kraus)
        outs.append(st.get_amps())
        st.close()
    scale = float(np.max(np.abs(rho)))
    assert float(np.max(np.abs(outs[0] - want))) <= 2.0 ** -48 * scale
    assert float(np.max(np.abs(outs[0] - outs[1]))) <= 2.0 ** -47 * scale


@pytest.mark.parametrize("nq", [9, 13, 21])
@pytest.mark.parametrize("arith", ["fx", "df"])
def test_dense_block_two_targets_on_tensor_cores(qs, nq, arith):
    """qs_apply_dense_block keeps two-target blocks on the tensor-core
    kernels (13 qubits: fewer tiles than SMs, the single-CTA kernel; 21: the
    warp-specialised kernel)."""
    rng = np.random.default_rng(4400 + nq + len(arith))
    psi = wl.random_statevector(nq, rng)
    mat = wl.haar_unitary(4, rng)
    targs = [int(x) for x in rng.choice(nq, 2, replace=False)]
    want = orc.apply_ctrl_multi_target(psi, [], targs, mat)
    st = fx_state(qs, nq, arith=qs.QS_ARITH_FX if arith == "fx" else qs.QS_ARITH_DF)
    st.set_amps(psi)
    qs.qs_apply_dense_block(st.handle, targs, mat)
    qs.qs_synchronize(st.handle)
    got = st.get_amps()
    st.close()
    ex = -51 if arith == "fx" else -44
    bound = 2.0 ** ex * (float(np.abs(mat).max()) * 4 * float(np.max(np.abs(psi))))
    assert float(np.max(np.abs(got - want))) <= bound
