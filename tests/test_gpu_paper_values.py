"""The whole solver against permeabilities the paper prints: the quadrant of the cubic sphere array
(Sec. 4.2, Table 3; 200 x 100 x 100 voxels, porosity 0.75, specular lateral faces, 8^3 velocities
below Kn = 1 and 16^3 from Kn = 1) converged to Err < 1e-6 at full size.  The paper's solver
differs in details it does not print, so agreement is tested to 5 %."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.mark.parametrize("kn", [0.1, 1.0])
def test_sphere_array_permeability_matches_table_3(kn):
    table = json.load(open(GOLDEN))["sphere_array_permeability"]
    k_paper = dict(zip(table["kn"], table["k"]))[kn]
    mask = inputs.sphere_quadrant(200, 100, 100, porosity=0.75)
    v, w = dvm.dvm_gh_velocity_grid(3, 8 if kn < 1 else 16)
    s = dvm.Solver(mask, kn, v, w, precision="fp32", lateral="specular", check_interval=100)
    st, it, err = s.iterate(3000, 1e-6)
    assert st == dvm.DVM_OK
    k, _ = s.permeability()
    print("Kn %g: %d iterations, k = %.5e, paper %.5e" % (kn, it, k, k_paper))
    assert abs(k / k_paper - 1) < 0.05
