"""The Python binding's own checks, on the CPU: option names and enum
names are validated before anything reaches the library, and image
arguments must be 2-D float32 CUDA tensors with unit column stride."""
import pytest

torch = pytest.importorskip("torch")

from paper_1203_5128_gb300 import api, build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


def test_options_by_name():
    o = api.bf_options_init(t_mode="tile", t_tile=128, plane_dtype="fp16", trunc_rule="chernoff",
                            filter="yvv", n_max=100)
    assert (o.t_mode, o.t_tile, o.plane_dtype, o.filter, o.n_max) == (
        api.T_MODES["tile"], 128, api.PLANES["fp16"], api.FILTERS["yvv"], 100)
    assert o.trunc_rule == api.RULES["chernoff"]
    d = api.bf_options_init()
    assert (d.t_mode, d.t_tile, d.n_max) == (api.T_MODES["global"], 64, 4096)
    assert d.spatial == api.SPATIALS["gauss"]
    assert api.bf_options_init(spatial="box").spatial == api.SPATIALS["box"]


def test_unknown_option_name_is_an_error():
    with pytest.raises(TypeError):
        api.bf_options_init(t_tiles=128)
    with pytest.raises(TypeError):
        api.bf_plan(64, 64, 2.0, 20.0, 0.01, planes="fp16")


def test_unknown_enum_name_is_an_error():
    with pytest.raises(ValueError):
        api.bf_options_init(t_mode="tiles")
    with pytest.raises(ValueError):
        api.bf_options_init(plane_dtype="fp8")
    with pytest.raises(ValueError):
        api.bf_options_init(spatial="disk")


@pytest.mark.parametrize("bad", [
    torch.zeros(8, 8),                                  # host memory
    torch.zeros(2, 8, 8),                               # not 2-D
    torch.zeros(8, 8, dtype=torch.float64),             # not float32
])
def test_image_checks(bad):
    with pytest.raises(ValueError):
        api._check_image(bad, "f")
