"""The debugging picture of a snapshot (App. B.1 BoardStrs), on the CPU."""
import oracle


def test_board_string_of_an_initial_position():
    import paper_2511_07312_gb300 as st
    pos = oracle.initial_position(oracle.setup_types(1, 0))
    text = st.board_string(pos)
    rows = text.splitlines()
    assert len(rows) == 11 and rows[-1] == "ply 0, red to move"
    cells = [c for r in rows[:10] for c in r.split()]
    assert len(cells) == 100
    assert cells.count("~~") == 8 and cells.count("..") == 12
    assert sum(c.startswith("r") for c in cells) == 40 and sum(c.startswith("b") for c in cells) == 40
    # rank 10 is printed first: blue's back row, then red's back row last
    assert all(c.startswith("b") for c in rows[0].split()) and all(c.startswith("r") for c in rows[9].split())
    assert sum(c.endswith("F") for c in cells) == 2 and sum(c.endswith("B") for c in cells) == 12
