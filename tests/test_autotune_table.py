"""The tuned-options table (paper_1612_04846_gb300/autotune.py) on the CPU: its JSON round trip and the
lookup of a class's options (the timing itself runs in the library's bura_autotune, on a GPU)."""
import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_1612_04846_gb300 import autotune, build_lib, bura
    build_lib.build(verbose=False)
    return autotune, bura


def test_table_round_trip_and_lookup(mods, tmp_path):
    autotune, bura = mods
    o = bura.bura_default_options()
    o.smoother_degree = 3
    o.smoother_ratio = 8.0
    o.sweeps = bura.BURA_SWEEP_GRID
    table = {"127x127:7": {"grid": [127, 127], "k": 7, "alpha": 0.5, "ms": 0.4,
                           "options": {f: getattr(o, f) for f, _ in bura.bura_options._fields_}}}
    path = str(tmp_path / "tuned.json")
    autotune.save(table, path)
    back = autotune.load(path)
    assert back == table
    got = autotune.options_for(back, (127, 127), 7)
    assert got.smoother_degree == 3 and got.smoother_ratio == 8.0 and got.sweeps == bura.BURA_SWEEP_GRID
    dflt = autotune.options_for(back, (255, 255), 7)  # not tuned: the defaults
    ref = bura.bura_default_options()
    assert all(getattr(dflt, f) == getattr(ref, f) for f, _ in bura.bura_options._fields_)


def test_autotune_rejects_bad_arguments_on_the_host(mods):
    _, bura = mods
    with pytest.raises(bura.BuraError) as ei:
        bura.bura_autotune((127, 127), 1.5, 7)
    assert ei.value.code == bura.BURA_EINVAL
    with pytest.raises(bura.BuraError) as ei:
        bura.bura_autotune((127, 127), 0.5, 7, trials=0)
    assert ei.value.code == bura.BURA_EINVAL
