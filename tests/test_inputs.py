"""The seeded input generator: determinism, symmetry O^{pq} = O^{qp}, consistency of the two views."""
import numpy as np

from paper_2305_15955_gb300 import inputs


def test_deterministic_and_seeded():
    spec = inputs.custom_system(30, 4, 50, seed=11)
    B1, B2 = inputs.build_B(spec), inputs.build_B(spec)
    assert np.array_equal(B1, B2)
    other = inputs.custom_system(30, 4, 50, seed=12)
    assert not np.allclose(B1, inputs.build_B(other))


def test_views_agree_and_symmetry():
    spec = inputs.custom_system(25, 5, 40, seed=3, n_core=2, states=(0, 1, 4), core_scale=0.3)
    B = inputs.build_B(spec)
    On = inputs.build_On(spec)
    nv = spec.n_virt
    for s, n in enumerate(spec.states):
        if n < spec.n_occ:
            assert np.array_equal(On[s][:, spec.n_occ:], B[:, n * nv:(n + 1) * nv])
    # O^{0,1} = O^{1,0}
    assert np.array_equal(On[0][:, 1], On[1][:, 0])


def test_core_scaling_and_statistics():
    spec = inputs.custom_system(60, 6, 400, seed=5, n_core=1, core_scale=0.3)
    B = inputs.build_B(spec)
    nv = spec.n_virt
    core = B[:, :nv] * np.sqrt(spec.n_aux)
    rest = B[:, nv:] * np.sqrt(spec.n_aux)
    assert abs(rest.mean()) < 0.02 and abs(rest.std() - 1.0) < 0.02
    assert abs(core.std() - 0.3) < 0.01


def test_eigenvalue_layouts():
    e = inputs.eigenvalues(inputs.small_system())
    assert e[0] == -10.6 and np.allclose(e[1:5], np.linspace(-1.1, -0.3, 4)) and abs(e[-1] - 2.0) < 1e-12
    e = inputs.eigenvalues(inputs.acene_system())
    assert len(e) == 1200 and abs(e[0] + 10.61) < 1e-12 and abs(e[5] + 10.59) < 1e-12 and abs(e[119] + 0.25) < 1e-12
    assert abs(e[120] - 0.01) < 1e-15 and abs(e[-1] - 5.0) < 1e-12
    batch = inputs.batched_systems()
    assert len(batch) == 16 and all(200 <= s.n_basis <= 1500 for s in batch)
    assert len({s.n_basis for s in batch}) > 8
