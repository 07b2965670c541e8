"""Pins for the synthetic workload definitions (closed forms and mesh validity)."""
import numpy as np

from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def test_star_solution_solves_poisson_and_is_continuous():
    h = 1e-4
    for r0 in (0.2, 0.45, 0.55, 0.8, 1.3, 3.0):
        for dirv in (np.array([1.0, 0, 0]), np.array([0.3, 0.4, np.sqrt(0.75)])):
            p0 = (r0 * dirv / np.linalg.norm(dirv))[None]
            lap = sum((inputs.star_solution(p0 + h * e) + inputs.star_solution(p0 - h * e)
                       - 2 * inputs.star_solution(p0)) / h ** 2 for e in np.eye(3))
            assert abs(-lap[0] - inputs.star_source(p0)[0]) < 2e-4 * max(1.0, inputs.star_source(p0)[0])
    for rj in (0.5, 1.0):   # value and radial derivative continuous across the jumps
        a = inputs.star_solution(np.array([[rj - 1e-9, 0, 0], [rj + 1e-9, 0, 0]]))
        assert abs(a[0] - a[1]) < 1e-7
        d1 = (inputs.star_solution(np.array([[rj - 1e-6, 0, 0]])) - inputs.star_solution(np.array([[rj - 2e-6, 0, 0]]))) / 1e-6
        d2 = (inputs.star_solution(np.array([[rj + 2e-6, 0, 0]])) - inputs.star_solution(np.array([[rj + 1e-6, 0, 0]]))) / 1e-6
        assert abs(d1[0] - d2[0]) < 1e-4
    # outside the star u = M / r with M the total "mass" int 4 pi rho r^2 dr
    M = 0.0
    for a, b in ((0.0, 0.5 - 1e-15), (0.5, 1.0 - 1e-15)):   # density is smooth on each piece
        s = np.linspace(a, b, 200001)
        M += np.trapezoid(4 * np.pi * inputs.star_density(s) * s * s, s)
    for r in (1.5, 4.0, 10.0):
        assert abs(inputs.star_solution(np.array([[r, 0, 0]]))[0] - M / r) < 1e-8


def test_workload_meshes_are_balanced_and_tile_the_box():
    for d in (inputs.star_mesh(), inputs.puncture_mesh(inputs.two_punctures()),
              inputs.puncture_mesh(inputs.three_punctures())):
        a, k = inputs.oracle_mesh_args(d)
        m = Mesh(*a, **k)             # raises on a 4:1 face or a hole
        vol = sum(np.prod(m.element_bounds(e)[1] - m.element_bounds(e)[0]) for e in range(m.n_elems))
        assert abs(vol - np.prod(np.asarray(d["hi"]) - np.asarray(d["lo"]))) < 1e-9 * vol
        assert d["p"].min() >= 1 and d["p"].max() <= 8


def test_three_punctures_triangle():
    pts = np.array([c for (_, c, _) in inputs.three_punctures()])
    sides = [np.linalg.norm(pts[i] - pts[(i + 1) % 3]) for i in range(3)]
    assert np.allclose(sides, 6.0, atol=1e-9)
    assert all(np.linalg.norm(P) <= 0.2 + 1e-12 for (_, _, P) in inputs.three_punctures())
