"""The launch table the autotuner writes and the library compiles in (host logic only)."""
import os

from paper_0805_1827_gb300 import autotune

TABLE = os.path.join(os.path.dirname(autotune.__file__), "csrc", "bap_tuning.inc")


def test_table_rows_are_well_formed():
    rows = autotune.read_table(TABLE)
    assert rows, "empty table"
    kinds = {r[1] for r in rows}
    assert kinds <= {0, 1} and 0 in kinds and 1 in kinds
    for d, kind, items, N, unit, ppl, t, share in rows:
        assert 1 <= d <= 10 and items > 0 and N > 0 and t > 0
        assert unit >= 32 and unit % 32 == 0 and unit <= 4096
        assert ppl in (1, 2) and (kind == 0 or ppl == 1)
        assert share in (1, 8)
    # one entry per shape
    keys = [(r[0], r[1], r[2], r[3]) for r in rows]
    assert len(keys) == len(set(keys))


def test_table_round_trips(tmp_path):
    rows = autotune.read_table(TABLE)
    out = tmp_path / "t.inc"
    autotune.write_table(rows, str(out))
    assert autotune.read_table(str(out)) == rows
